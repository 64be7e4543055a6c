"""Thin ctypes binding over the C ABI of include/lbm.h (argument marshalling only).

Every step of the method runs in the CUDA library ``libtslb_b300.so``; this module only converts
arguments.  Host arrays are numpy float32; device arrays are torch CUDA float32 tensors (torch
provides device memory and the stream, nothing else).  There is no CPU fallback: if the library
is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtslb_b300.so")

LBM_OK = 0
LBM_FP32, LBM_BF16, LBM_FP16 = 0, 1, 2     # lbm_storage: population storage formats
LBM_MOM = 3                                 # lbm_storage: moment-only storage (p*, u, a, B per node)
LBM_MOM_BF16, LBM_MOM_FP16 = 4, 5           # ... with a and B stored in BF16 / FP16
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA",
          -4: "LBM_ERR_NONFINITE", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE"}


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_size_t),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_z", ctypes.c_int),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("mu_l", ctypes.c_double), ("mu_g", ctypes.c_double),
        ("sigma", ctypes.c_double), ("width", ctypes.c_double), ("mobility", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("rho_ref", ctypes.c_double),
        ("body", ctypes.c_double * 3),
        ("storage", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


class LbmObs(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_double), ("sum_phi", ctypes.c_double), ("mass", ctypes.c_double),
        ("sum_pstar", ctypes.c_double),
        ("momentum", ctypes.c_double * 3),
        ("centroid_liq", ctypes.c_double * 3), ("centroid_gas", ctypes.c_double * 3),
        ("vel_liq", ctypes.c_double * 3), ("vel_gas", ctypes.c_double * 3),
        ("p_liq", ctypes.c_double), ("p_gas", ctypes.c_double),
        ("n_liq", ctypes.c_double), ("n_gas", ctypes.c_double),
        ("umax", ctypes.c_double), ("phi_min", ctypes.c_double), ("phi_max", ctypes.c_double),
        ("n_nonfinite", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else float(v)
        return out


class LbmTuning(ctypes.Structure):
    """Launch configuration of the ensemble kernels (lbm_tuning)."""
    _fields_ = [("lbm_block", ctypes.c_int), ("ac_rows", ctypes.c_int), ("ac_zlen", ctypes.c_int),
                ("graph_steps", ctypes.c_int), ("lbm_us", ctypes.c_double), ("ac_us", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class LbmClosureNorm(ctypes.Structure):
    """Input normalisation and correction scales of the learned closure (lbm_closure_norm)."""
    _fields_ = [("in_shift", ctypes.c_float * 5), ("in_scale", ctypes.c_float * 5),
                ("out_scale", ctypes.c_float * 4)]

    @classmethod
    def make(cls, in_shift, in_scale, out_scale):
        n = cls()
        n.in_shift[:] = [float(v) for v in in_shift]
        n.in_scale[:] = [float(v) for v in in_scale]
        n.out_scale[:] = [float(v) for v in out_scale]
        return n


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with paper_2501_00846_b300.build.build()")
    L = ctypes.CDLL(path)
    vp, i, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    fp = ctypes.c_void_p
    sigs = {
        "lbm_create": ([ctypes.POINTER(LbmParams), ctypes.POINTER(vp)], i),
        "lbm_init_fields": ([vp, fp, fp, fp, i], i),
        "lbm_step": ([vp, i], i),
        "lbm_observables": ([vp, ctypes.POINTER(LbmObs)], i),
        "lbm_read_fields": ([vp, fp, fp, fp, i], i),
        "lbm_get_state": ([vp, fp, fp, fp, i], i),
        "lbm_set_state": ([vp, fp, fp, fp, ll, i], i),
        "lbm_synchronize": ([vp], i),
        "lbm_num_nodes": ([vp], ll),
        "lbm_step_count": ([vp], ll),
        "lbm_set_path": ([vp, i], i),
        "lbm_set_split": ([vp, i], i),
        "lbm_set_advection": ([vp, i], i),
        "lbm_run_phase": ([vp, i, i], i),
        "lbm_destroy": ([vp], None),
        "lbm_status_string": ([i], ctypes.c_char_p),
        "lbm_last_error": ([], ctypes.c_char_p),
        "lbm_abi_version": ([], i),
        "lbm_observables_noalloc": ([fp, fp, fp, i, i, i, ctypes.c_double, ctypes.c_double, vp,
                                     ctypes.POINTER(LbmObs)], i),
        "lbm_ens_create": ([ctypes.POINTER(LbmParams), i, vp, ctypes.POINTER(vp)], i),
        "lbm_ens_destroy": ([vp], None),
        "lbm_ens_init_fields": ([vp, i, fp, fp, fp, i], i),
        "lbm_ens_step": ([vp, i], i),
        "lbm_ens_observables": ([vp, i, ctypes.POINTER(LbmObs)], i),
        "lbm_ens_read_fields": ([vp, i, fp, fp, fp, i], i),
        "lbm_ens_get_tuning": ([vp, ctypes.POINTER(LbmTuning)], i),
        "lbm_ens_set_tuning": ([vp, ctypes.POINTER(LbmTuning)], i),
        "lbm_ens_autotune": ([vp, i, ctypes.POINTER(LbmTuning)], i),
        "lbm_ens_num_boxes": ([vp], i),
        "lbm_ens_num_nodes": ([vp], ll),
        "lbm_ens_box_nodes": ([vp, i], ll),
        "lbm_ens_step_count": ([vp], ll),
        "lbm_ens_restrict_state": ([vp, i, vp], i),
        "lbm_ens_set_persistent": ([vp, i], i),
        "lbm_ens_test_stall_barrier": ([vp, i], i),
        "lbm_cnn_create": ([i, i, i, ctypes.c_ulonglong, vp, ctypes.POINTER(vp)], i),
        "lbm_cnn_destroy": ([vp], None),
        "lbm_cnn_num_params": ([], i),
        "lbm_cnn_get_params": ([vp, fp], i),
        "lbm_cnn_set_params": ([vp, fp], i),
        "lbm_cnn_get_grads": ([vp, fp], i),
        "lbm_cnn_get_layer": ([vp, i, fp, fp, fp], i),
        "lbm_cnn_forward": ([vp, fp, fp], i),
        "lbm_cnn_set_conv_kernel": ([vp, i], i),
        "lbm_cnn_test_expire_wait": ([vp, i], i),
        "lbm_cnn_grad": ([vp, fp, fp, i, ctypes.POINTER(ctypes.c_double)], i),
        "lbm_cnn_adam_step": ([vp, ctypes.c_float, ctypes.c_float], i),
        "lbm_closure_features": ([vp, ctypes.POINTER(LbmClosureNorm), fp], i),
        "lbm_closure_target": ([vp, fp, ctypes.POINTER(LbmClosureNorm), fp], i),
        "lbm_closure_apply": ([vp, vp, ctypes.POINTER(LbmClosureNorm)], i),
        "lbm_restrict2": ([fp, fp, fp, i, i, i, ctypes.c_double, ctypes.c_double, fp, vp], i),
        "lbm_prolong2_state": ([vp, vp], i),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status: int):
    if status != LBM_OK:
        raise LbmError(status, load().lbm_last_error().decode())


def make_params(nx, ny, nz, wall_z=0, rho_l=1.0, rho_g=0.1, mu_l=0.1, mu_g=0.01, sigma=0.01,
                width=4.0, mobility=0.1, gravity=(0.0, 0.0, 0.0), rho_ref=1.0,
                body=(0.0, 0.0, 0.0), storage=0, stream=None) -> LbmParams:
    p = LbmParams()
    p.struct_size = ctypes.sizeof(LbmParams)
    p.nx, p.ny, p.nz, p.wall_z = int(nx), int(ny), int(nz), int(wall_z)
    p.rho_l, p.rho_g, p.mu_l, p.mu_g = rho_l, rho_g, mu_l, mu_g
    p.sigma, p.width, p.mobility = sigma, width, mobility
    p.gravity[:] = [float(v) for v in gravity]
    p.rho_ref = rho_ref
    p.body[:] = [float(v) for v in body]
    p.storage = int(storage)
    p.stream = stream
    return p


def _ptr(a, n: int, writable: bool):
    """(pointer, on_device) of a float32 numpy array or torch CUDA tensor with n elements."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous or a.size != n:
            raise ValueError(f"expected a C-contiguous float32 array of {n} elements")
        if writable and not a.flags.writeable:
            raise ValueError("output array is read-only")
        return a.ctypes.data, 0
    import torch
    if not isinstance(a, torch.Tensor) or not a.is_cuda or a.dtype != torch.float32 \
            or not a.is_contiguous() or a.numel() != n:
        raise ValueError(f"expected a contiguous float32 CUDA tensor of {n} elements")
    return a.data_ptr(), 1


class Solver:
    """One box on the current CUDA device, driven through the C ABI.

    ``stream``: a ``torch.cuda.Stream`` (default: torch's current stream at construction)."""

    def __init__(self, stream=None, **params):
        import torch
        L = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.params = make_params(stream=stream.cuda_stream, **params)
        self._ctx = ctypes.c_void_p()
        _check(L.lbm_create(ctypes.byref(self.params), ctypes.byref(self._ctx)))
        self.shape = (self.params.nz, self.params.ny, self.params.nx)
        self.n = int(L.lbm_num_nodes(self._ctx))

    # -- lifecycle --------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            load().lbm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls ------------------------------------------------------------------------------
    def init_fields(self, phi, u, pstar=None):
        pp, d1 = _ptr(phi, self.n, False)
        up, d2 = _ptr(u, 3 * self.n, False)
        sp, d3 = _ptr(pstar, self.n, False)
        on_dev = {d for d in (d1, d2, d3) if d is not None}
        if len(on_dev) != 1:
            raise ValueError("inputs must all be host arrays or all device tensors")
        _check(load().lbm_init_fields(self._ctx, pp, up, sp, on_dev.pop()))

    def step(self, nsteps: int = 1):
        _check(load().lbm_step(self._ctx, int(nsteps)))

    def synchronize(self):
        _check(load().lbm_synchronize(self._ctx))

    def set_path(self, path: int):
        _check(load().lbm_set_path(self._ctx, int(path)))

    def set_advection(self, form: int):
        """0: flux form div(ubar phi) (default); 1: literal ubar . grad(phi), path 1 only."""
        _check(load().lbm_set_advection(self._ctx, int(form)))

    def set_split(self, split: int):
        """z chunks per column tile of the marching kernels (paths 0 and 2); 0 = default."""
        _check(load().lbm_set_split(self._ctx, int(split)))

    def run_phase(self, phase: int, nrep: int = 1):
        """Launch one kernel of the two-kernel step nrep times without advancing the state."""
        _check(load().lbm_run_phase(self._ctx, int(phase), int(nrep)))

    @property
    def step_count(self) -> int:
        return int(load().lbm_step_count(self._ctx))

    def observables(self, allow_nonfinite: bool = False) -> dict:
        o = LbmObs()
        st = load().lbm_observables(self._ctx, ctypes.byref(o))
        if st == -4 and allow_nonfinite:
            return o.as_dict()
        _check(st)
        return o.as_dict()

    def read_fields(self, phi=None, u=None, p=None):
        """Fill the given outputs (numpy or CUDA tensors); with no argument return host copies
        (phi[nz,ny,nx], u[3,nz,ny,nx], p[nz,ny,nx])."""
        if phi is None and u is None and p is None:
            phi = np.empty(self.shape, np.float32)
            u = np.empty((3,) + self.shape, np.float32)
            p = np.empty(self.shape, np.float32)
        ptrs = [_ptr(phi, self.n, True), _ptr(u, 3 * self.n, True), _ptr(p, self.n, True)]
        on_dev = {d for _, d in ptrs if d is not None}
        if len(on_dev) != 1:
            raise ValueError("outputs must all be host arrays or all device tensors")
        _check(load().lbm_read_fields(self._ctx, ptrs[0][0], ptrs[1][0], ptrs[2][0], on_dev.pop()))
        return phi, u, p

    def get_state(self):
        g = np.empty((27,) + self.shape, np.float32)
        phi = np.empty(self.shape, np.float32)
        u = np.empty((3,) + self.shape, np.float32)
        _check(load().lbm_get_state(self._ctx, g.ctypes.data, phi.ctypes.data, u.ctypes.data, 0))
        return g, phi, u

    def set_state(self, g, phi, u, step: int = 0):
        gp, d1 = _ptr(g, 27 * self.n, False)
        pp, d2 = _ptr(phi, self.n, False)
        up, d3 = _ptr(u, 3 * self.n, False)
        on_dev = {d1, d2, d3}
        if len(on_dev) != 1:
            raise ValueError("inputs must all be host arrays or all device tensors")
        _check(load().lbm_set_state(self._ctx, gp, pp, up, int(step), on_dev.pop()))


def from_workload(wl, stream=None, storage: int = LBM_FP32) -> Solver:
    """Solver for an inputs.Workload, initialised with its seeded phi0, u0 and p*0 (FP64 -> FP32).
    ``storage``: LBM_FP32, LBM_BF16 or LBM_FP16 population storage, or LBM_MOM, LBM_MOM_BF16 or
    LBM_MOM_FP16 moment storage."""
    s = Solver(stream=stream, storage=storage, **wl.params())
    ps = wl.pstar_init()
    s.init_fields(np.ascontiguousarray(wl.phi0(), np.float32), np.ascontiguousarray(wl.u0(), np.float32),
                  None if ps is None else np.ascontiguousarray(ps, np.float32))
    return s


class Ensemble:
    """Independent boxes advanced together by the batched kernels (lbm_ens_* of the C ABI).

    ``boxes``: a list of parameter dicts (keyword arguments of make_params, e.g. Workload.params());
    ``stream``: a torch.cuda.Stream (default: torch's current stream at construction)."""

    def __init__(self, boxes, stream=None):
        import torch
        L = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        arr = (LbmParams * len(boxes))()
        for b, prm in enumerate(boxes):
            arr[b] = make_params(stream=None, **prm)
        self._params = arr
        self._ens = ctypes.c_void_p()
        _check(L.lbm_ens_create(arr, len(boxes), stream.cuda_stream, ctypes.byref(self._ens)))
        self.nboxes = len(boxes)
        self.shapes = [(p.nz, p.ny, p.nx) for p in arr]
        self.sizes = [int(L.lbm_ens_box_nodes(self._ens, b)) for b in range(self.nboxes)]
        self.n = int(L.lbm_ens_num_nodes(self._ens))

    def close(self):
        if getattr(self, "_ens", None) and self._ens.value:
            load().lbm_ens_destroy(self._ens)
            self._ens = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_fields(self, box: int, phi, u, pstar=None):
        n = self.sizes[box]
        pp, d1 = _ptr(phi, n, False)
        up, d2 = _ptr(u, 3 * n, False)
        sp, d3 = _ptr(pstar, n, False)
        on_dev = {d for d in (d1, d2, d3) if d is not None}
        if len(on_dev) != 1:
            raise ValueError("inputs must all be host arrays or all device tensors")
        _check(load().lbm_ens_init_fields(self._ens, int(box), pp, up, sp, on_dev.pop()))

    def step(self, nsteps: int = 1):
        _check(load().lbm_ens_step(self._ens, int(nsteps)))

    @property
    def step_count(self) -> int:
        return int(load().lbm_ens_step_count(self._ens))

    def observables(self, box: int, allow_nonfinite: bool = False) -> dict:
        o = LbmObs()
        st = load().lbm_ens_observables(self._ens, int(box), ctypes.byref(o))
        if st == -4 and allow_nonfinite:
            return o.as_dict()
        _check(st)
        return o.as_dict()

    def read_fields(self, box: int):
        """Host copies (phi[nz,ny,nx], u[3,nz,ny,nx], p[nz,ny,nx]) of one box."""
        shape = self.shapes[box]
        phi = np.empty(shape, np.float32)
        u = np.empty((3,) + shape, np.float32)
        p = np.empty(shape, np.float32)
        _check(load().lbm_ens_read_fields(self._ens, int(box), phi.ctypes.data, u.ctypes.data, p.ctypes.data, 0))
        return phi, u, p

    @property
    def tuning(self) -> dict:
        t = LbmTuning()
        _check(load().lbm_ens_get_tuning(self._ens, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = LbmTuning()
        _check(load().lbm_ens_get_tuning(self._ens, ctypes.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        _check(load().lbm_ens_set_tuning(self._ens, ctypes.byref(t)))

    def restrict_state(self, box: int, coarse: "Solver"):
        """Set a half-size context's state to the 2x restriction of box ``box``'s state."""
        _check(load().lbm_ens_restrict_state(self._ens, int(box), coarse._ctx))

    def autotune(self, reps: int = 5) -> dict:
        t = LbmTuning()
        _check(load().lbm_ens_autotune(self._ens, int(reps), ctypes.byref(t)))
        return t.as_dict()

    def set_persistent(self, on: bool):
        """One persistent cooperative launch per step (True) or two graph-replayed launches (False)."""
        _check(load().lbm_ens_set_persistent(self._ens, int(bool(on))))

    def test_stall_barrier(self, on: bool):
        """Test hook: make every grid-barrier wait of the persistent step expire (LBM_ERR_TIMEOUT)."""
        _check(load().lbm_ens_test_stall_barrier(self._ens, int(bool(on))))


def ensemble_from_workloads(workloads, stream=None, storage: int = LBM_FP32) -> Ensemble:
    """Ensemble of inputs.Workload boxes, each initialised with its seeded phi0, u0 and p*0.
    ``storage``: LBM_FP32 or one of the moment storages (the same for every box)."""
    e = Ensemble([dict(wl.params(), storage=storage) for wl in workloads], stream=stream)
    for b, wl in enumerate(workloads):
        ps = wl.pstar_init()
        e.init_fields(b, np.ascontiguousarray(wl.phi0(), np.float32), np.ascontiguousarray(wl.u0(), np.float32),
                      None if ps is None else np.ascontiguousarray(ps, np.float32))
    return e


# layer shapes of the closure network: (output channels, input channels)
CNN_LAYERS = [(32, 5), (32, 32), (32, 32), (4, 32)]


def _dev(t, n):
    """Device pointer of a contiguous float32 CUDA tensor with n elements."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() \
            or t.numel() != n:
        raise ValueError(f"expected a contiguous float32 CUDA tensor of {n} elements")
    return t.data_ptr()


class Network:
    """The learned closure's network (lbm_cnn_* of the C ABI) for nx x ny x nz periodic grids."""

    def __init__(self, nx, ny, nz, seed=0, stream=None):
        import torch
        L = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self._cnn = ctypes.c_void_p()
        _check(L.lbm_cnn_create(nx, ny, nz, int(seed), stream.cuda_stream, ctypes.byref(self._cnn)))
        self.num_params = int(L.lbm_cnn_num_params())

    def close(self):
        if getattr(self, "_cnn", None) and self._cnn.value:
            load().lbm_cnn_destroy(self._cnn)
            self._cnn = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, np.float32)
        _check(load().lbm_cnn_get_params(self._cnn, out.ctypes.data))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        if flat.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters")
        _check(load().lbm_cnn_set_params(self._cnn, flat.ctypes.data))

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.num_params, np.float32)
        _check(load().lbm_cnn_get_grads(self._cnn, out.ctypes.data))
        return out

    def get_layer(self, layer: int):
        """(a_in [CIN][nz, ny, nx], z [COUT][...], dz [COUT][...]) of layer 0..3 as FP32 host arrays:
        the layer's BF16 input widened to FP32, its pre-activation from the last forward or grad
        call, and d loss / d z from the last grad call."""
        cout, cin = CNN_LAYERS[layer]
        a = np.empty((cin,) + self.shape, np.float32)
        z = np.empty((cout,) + self.shape, np.float32)
        dz = np.empty((cout,) + self.shape, np.float32)
        _check(load().lbm_cnn_get_layer(self._cnn, int(layer), a.ctypes.data, z.ctypes.data, dz.ctypes.data))
        return a, z, dz

    @staticmethod
    def split(flat):
        """[(W [cout, cin, 27], b [cout]) per layer] views of a flat parameter vector."""
        out, o = [], 0
        for cout, cin in CNN_LAYERS:
            w = flat[o:o + cout * cin * 27].reshape(cout, cin, 27)
            o += cout * cin * 27
            out.append((w, flat[o:o + cout]))
            o += cout
        return out

    def test_expire_wait(self, on: bool):
        """Test hook: make the tensor-core convolutions' waits expire (LBM_ERR_TIMEOUT)."""
        _check(load().lbm_cnn_test_expire_wait(self._cnn, int(bool(on))))

    def set_conv_kernel(self, kernel: int):
        """0: tcgen05 with TMEM accumulators; 1: mma.sync from shared-memory tiles (default);
        2: mma.sync with fragments straight from global memory."""
        _check(load().lbm_cnn_set_conv_kernel(self._cnn, int(kernel)))

    def forward(self, x, y):
        _check(load().lbm_cnn_forward(self._cnn, _dev(x, 5 * self.n), _dev(y, 4 * self.n)))

    def grad(self, x, t, accumulate=False) -> float:
        loss = ctypes.c_double()
        _check(load().lbm_cnn_grad(self._cnn, _dev(x, 5 * self.n), _dev(t, 4 * self.n), int(bool(accumulate)),
                                   ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr, grad_scale=1.0):
        _check(load().lbm_cnn_adam_step(self._cnn, float(lr), float(grad_scale)))


def closure_features(s: "Solver", norm: LbmClosureNorm, x):
    _check(load().lbm_closure_features(s._ctx, ctypes.byref(norm), _dev(x, 5 * s.n)))


def closure_target(s: "Solver", ref, norm: LbmClosureNorm, t):
    import torch
    if not isinstance(ref, torch.Tensor) or not ref.is_cuda or ref.dtype != torch.float32 or not ref.is_contiguous() \
            or ref.numel() < 4 * s.n:
        raise ValueError("ref must be a contiguous float32 CUDA tensor of at least 4 N elements")
    _check(load().lbm_closure_target(s._ctx, ref.data_ptr(), ctypes.byref(norm), _dev(t, 4 * s.n)))


def closure_apply(s: "Solver", net: Network, norm: LbmClosureNorm):
    _check(load().lbm_closure_apply(s._ctx, net._cnn, ctypes.byref(norm)))


def restrict2(phi, u, p, nx, ny, nz, rho_l, rho_g, out, stream=None):
    """Coarse (phi, u, p, p*) [6][N/8] of a fine state (device tensors, channel-first)."""
    import torch
    n = nx * ny * nz
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(load().lbm_restrict2(_dev(phi, n), _dev(u, 3 * n), _dev(p, n), nx, ny, nz, float(rho_l), float(rho_g),
                                _dev(out, 6 * (n // 8)), st))


def prolong2_state(coarse: "Solver", fine: "Solver"):
    """Set fine's state to the 2x cell-centred prolongation of coarse's (lbm_prolong2_state)."""
    _check(load().lbm_prolong2_state(coarse._ctx, fine._ctx))
