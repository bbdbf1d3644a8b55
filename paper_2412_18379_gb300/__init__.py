"""GB300 particle location for the CNN-SNS method (thin Python binding).

Every step of the path runs in libcnnsns.so (CUDA kernels for sm_103a + host
C++); this module only marshals arguments: numpy arrays for host inputs,
torch CUDA tensors for device memory and streams.
"""

import ctypes

import numpy as np

from . import _capi
from ._capi import (CS_SNS, CS_CNN_SNS, CS_ASG_DIRECT, CS_FOUND, CS_OUTSIDE,
                    CS_FOUND_VIA_FALLBACK, CS_INVALID, CS_EPS, CS_NO_FIELD, CsError)

MODES = {"sns": CS_SNS, "cnn": CS_CNN_SNS, "cnn_sns": CS_CNN_SNS, "asg": CS_ASG_DIRECT,
         "asg_direct": CS_ASG_DIRECT}

__all__ = ["Context", "Mesh", "Field", "CsError", "CS_SNS", "CS_CNN_SNS", "CS_ASG_DIRECT",
           "CS_FOUND", "CS_OUTSIDE", "CS_FOUND_VIA_FALLBACK", "CS_INVALID", "CS_EPS",
           "CS_NO_FIELD", "check_track_args"]


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream)


_DTYPE_NAMES = {}


def _dtype_name(a):
    d = a.dtype
    name = _DTYPE_NAMES.get(d)
    if name is None:
        name = _DTYPE_NAMES[d] = str(d).replace("torch.", "")
    return name


def _numel(a):
    """Element count of a numpy array or a torch tensor."""
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _contiguous(a):
    if isinstance(a, np.ndarray):
        return a.flags["C_CONTIGUOUS"]
    return a.is_contiguous()


def check_track_args(dim, x, u, start=None, out=None, on_device=True):
    """Check the arrays of a tracking call before any pointer reaches the C
    ABI, which trusts the sizes it is given: a wrong dtype, shape or stride
    would make the kernels read or write past the arrays. x, u: contiguous
    float64 [n, dim]; start: contiguous int32 [n]; out: contiguous host,
    path_len (int32), status (uint8) and start (int32) with at least n
    elements. on_device: every array must be a CUDA tensor on x's device
    (else CPU memory). Raises ValueError; returns n."""
    if getattr(x, "ndim", None) != 2 or x.shape[1] != dim:
        raise ValueError("x must have shape [n, %d]" % dim)
    n = int(x.shape[0])
    arrays = [("x", x, "float64", (n, dim)), ("u", u, "float64", (n, dim))]
    if start is not None:
        arrays.append(("start", start, "int32", (n,)))
    for key, dt in (("host", "int32"), ("path_len", "int32"), ("status", "uint8"),
                    ("start", "int32")):
        if out is not None and out.get(key) is not None:
            arrays.append(("out['%s']" % key, out[key], dt, None))
    dev = getattr(x, "device", None)
    for name, a, dt, shape in arrays:
        if a is None:
            raise ValueError("%s is missing" % name)
        if _dtype_name(a) != dt:
            raise ValueError("%s must be %s, not %s" % (name, dt, _dtype_name(a)))
        if not _contiguous(a):
            raise ValueError("%s must be contiguous" % name)
        if shape is not None and tuple(a.shape) != shape:
            raise ValueError("%s must have shape %s, not %s" % (name, shape, tuple(a.shape)))
        if shape is None and _numel(a) < n:
            raise ValueError("%s holds %d elements, fewer than n = %d" % (name, _numel(a), n))
        cuda = bool(getattr(a, "is_cuda", False))
        if on_device and (not cuda or a.device != dev):
            raise ValueError("%s must be a CUDA tensor on %s" % (name, dev))
        if not on_device and cuda:
            raise ValueError("%s must be in host memory" % name)
    return n


def _check_dev(name, a, dtype, shape, device=None):
    """A contiguous CUDA tensor of the given dtype and shape (None: any
    extent on that axis), on `device` if given. Raises ValueError."""
    if a is None:
        raise ValueError("%s is missing" % name)
    if not getattr(a, "is_cuda", False):
        raise ValueError("%s must be a CUDA tensor" % name)
    if device is not None and a.device != device:
        raise ValueError("%s must be on %s" % (name, device))
    if _dtype_name(a) != dtype:
        raise ValueError("%s must be %s, not %s" % (name, dtype, _dtype_name(a)))
    if not _contiguous(a):
        raise ValueError("%s must be contiguous" % name)
    if a.ndim != len(shape) or any(s is not None and a.shape[i] != s
                                   for i, s in enumerate(shape)):
        raise ValueError("%s must have shape %s, not %s"
                         % (name, tuple("n" if s is None else s for s in shape),
                            tuple(a.shape)))


class Mesh:
    def __init__(self, ctx, mesh_id, dim, n_v, n_e):
        self.ctx = ctx
        self.id = mesh_id
        self.dim = dim
        self.n_vertices = n_v
        self.n_elements = n_e

    def info(self):
        inf = _capi.MeshInfo()
        self.ctx._check(self.ctx.lib.cs_mesh_query(self.ctx.h, self.id, ctypes.byref(inf)))
        d = inf.dim
        return dict(dim=d, n_vertices=inf.n_vertices, n_elements=inf.n_elements,
                    asg_grid=list(inf.asg_grid[:d]), bucket_grid=list(inf.bucket_grid[:d]),
                    bucket_items=inf.bucket_items, lo=list(inf.lo[:d]), hi=list(inf.hi[:d]),
                    tau=inf.tau, step_cap=inf.step_cap, record_bytes=inf.record_bytes,
                    device_bytes=inf.device_bytes, pred_stride=inf.pred_stride,
                    pred_grid=list(inf.pred_grid[:d]))

    def set_predictor_grid(self, stride):
        """Run the start predictor on cells of stride^dim ASG cells (odd
        stride; 1 = the ASG grid). Drops the stored grid velocity."""
        self.ctx._check(self.ctx.lib.cs_predictor_grid(self.ctx.h, self.id, int(stride)))

    def node_start_elements(self):
        out = np.empty(self.n_vertices, dtype=np.int32)
        self.ctx._check(self.ctx.lib.cs_node_start_elements(self.ctx.h, self.id, _ptr(out)))
        return out

    def seed_grid(self):
        g = self.info()["asg_grid"]
        out = np.empty(int(np.prod(g)), dtype=np.int32)
        self.ctx._check(self.ctx.lib.cs_seed_grid(self.ctx.h, self.id, _ptr(out)))
        return out

    def release(self):
        if self.id is not None:
            self.ctx._check(self.ctx.lib.cs_mesh_release(self.ctx.h, self.id))
            self.id = None


class Field:
    """A velocity field of a mesh, resident on the device (cs_field_upload)."""

    def __init__(self, ctx, field_id, mesh):
        self.ctx = ctx
        self.id = field_id
        self.mesh = mesh

    def release(self):
        if self.id is not None:
            self.ctx._check(self.ctx.lib.cs_field_release(self.ctx.h, self.id))
            self.id = None


def _field_id(field):
    if field is None:
        return CS_NO_FIELD
    return field.id if isinstance(field, Field) else int(field)


class Context:
    """One library context on one CUDA device; hbm_budget caps the device
    bytes it may hold (0 = no cap)."""

    def __init__(self, device=0, hbm_budget=0, lib_path=None):
        self.lib = _capi.load(lib_path)
        h = ctypes.c_void_p()
        rc = self.lib.cs_create(ctypes.byref(h), int(device), int(hbm_budget))
        if rc != 0:
            raise CsError(rc, "cs_create(device=%d) failed" % device)
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.lib.cs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            msg = self.lib.cs_last_error(self.h)
            raise CsError(rc, msg.decode() if msg else "")

    @property
    def launches(self):
        return int(self.lib.cs_kernel_launches(self.h))

    def memory_usage(self):
        """(device bytes held, budget) of the context."""
        used, budget = ctypes.c_size_t(), ctypes.c_size_t()
        self._check(self.lib.cs_memory_usage(self.h, ctypes.byref(used), ctypes.byref(budget)))
        return int(used.value), int(budget.value)

    def upload_field(self, mesh, u_nodal):
        """Resident velocity field of a mesh from its nodal velocity [n_v, dim]
        (float64 numpy array or torch tensor, host or CUDA)."""
        if isinstance(u_nodal, np.ndarray):
            u_nodal = np.ascontiguousarray(u_nodal, dtype=np.float64)
        if (_dtype_name(u_nodal) != "float64" or not _contiguous(u_nodal)
                or tuple(u_nodal.shape) != (mesh.n_vertices, mesh.dim)):
            raise ValueError("u_nodal must be contiguous float64 [%d, %d]"
                             % (mesh.n_vertices, mesh.dim))
        fid = ctypes.c_int32()
        self._check(self.lib.cs_field_upload(self.h, mesh.id, _ptr(u_nodal), ctypes.byref(fid)))
        return Field(self, fid.value, mesh)

    def profile(self, on=True):
        self._check(self.lib.cs_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, reset=True):
        """{stage: (launches, total ms)} from CUDA events on the launch stream."""
        p = _capi.Profile()
        self._check(self.lib.cs_profile_read(self.h, ctypes.byref(p), 1 if reset else 0))
        return {name: (int(p.launches[i]), float(p.ms[i]))
                for i, name in enumerate(_capi.STAGES)}

    def upload_mesh(self, xyz, conn, asg_grid=None):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        dim = xyz.shape[1]
        if conn.shape[1] != dim + 1:
            raise ValueError("conn must have dim+1 columns")
        g = None
        if asg_grid is not None:
            g = np.ascontiguousarray(np.broadcast_to(np.asarray(asg_grid), (dim,)),
                                     dtype=np.int32)
        mid = ctypes.c_int32()
        self._check(self.lib.cs_mesh_upload(self.h, dim, xyz.shape[0], _ptr(xyz),
                                            conn.shape[0], _ptr(conn), _ptr(g),
                                            ctypes.byref(mid)))
        return Mesh(self, mid.value, dim, xyz.shape[0], conn.shape[0])

    def _device_out(self, n, dev, out, start_out):
        import torch
        if out is None:
            out = dict(host=torch.empty(n, dtype=torch.int32, device=dev),
                       path_len=torch.empty(n, dtype=torch.int32, device=dev),
                       status=torch.empty(n, dtype=torch.uint8, device=dev))
            if start_out:
                out["start"] = torch.empty(n, dtype=torch.int32, device=dev)
        return out

    def track(self, mesh, x, u, dt, start=None, mode="sns", out=None, start_out=False,
              stream=None, field=None):
        """Device path: x, u are float64 CUDA tensors [n, dim]; returns (or
        fills `out` with) device tensors host, path_len, status[, start].
        field: the Field (or id) whose grid velocity CNN-SNS predicts from."""
        import torch
        n = check_track_args(mesh.dim, x, u, start, out)
        out = self._device_out(n, x.device, out, start_out)
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        self._check(self.lib.cs_track(
            self.h, mesh.id, _field_id(field), n, _ptr(x), _ptr(u), float(dt), _ptr(start),
            MODES[mode] if isinstance(mode, str) else int(mode), _ptr(out["host"]),
            _ptr(out["path_len"]), _ptr(out["status"]), _ptr(out.get("start")),
            _stream_ptr(st)))
        return out

    def track_noalloc(self, mesh, x, u, dt, start=None, mode="sns", out=None, start_out=False,
                      stream=None, field=None):
        """cs_track_noalloc: like track(), but the library allocates nothing;
        pass `out` (preallocated device tensors) to keep the call allocation-
        free on this side too. Same n range as track(); CNN-SNS is refused."""
        import torch
        n = check_track_args(mesh.dim, x, u, start, out)
        out = self._device_out(n, x.device, out, start_out)
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        self._check(self.lib.cs_track_noalloc(
            self.h, mesh.id, _field_id(field), n, _ptr(x), _ptr(u), float(dt), _ptr(start),
            MODES[mode] if isinstance(mode, str) else int(mode), _ptr(out["host"]),
            _ptr(out["path_len"]), _ptr(out["status"]), _ptr(out.get("start")),
            _stream_ptr(st)))
        return out

    def track_host(self, mesh, x, u, dt, start=None, mode="sns", out=None, start_out=False,
                   field=None):
        """Host path: numpy (or pinned torch CPU) inputs; copies in, runs,
        copies out and synchronises inside the library."""
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
            u = np.ascontiguousarray(u, dtype=np.float64)
            if start is not None:
                start = np.ascontiguousarray(start, dtype=np.int32)
        # one check of every array; outputs made here need none
        n = check_track_args(mesh.dim, x, u, start, out, on_device=False)
        if out is None:
            out = dict(host=np.empty(n, dtype=np.int32), path_len=np.empty(n, dtype=np.int32),
                       status=np.empty(n, dtype=np.uint8))
            if start_out:
                out["start"] = np.empty(n, dtype=np.int32)
        self._check(self.lib.cs_track_host(
            self.h, mesh.id, _field_id(field), n, _ptr(x), _ptr(u), float(dt), _ptr(start),
            MODES[mode] if isinstance(mode, str) else int(mode), _ptr(out["host"]),
            _ptr(out["path_len"]), _ptr(out["status"]), _ptr(out.get("start"))))
        return out

    def track_nodes_host(self, mesh, u, dt, mode="sns", out=None, start_out=False, field=None):
        """track_host for the mesh nodes at their uploaded coordinates: only
        u (host float64 [n_v, dim]) is copied in."""
        if isinstance(u, np.ndarray):
            u = np.ascontiguousarray(u, dtype=np.float64)
        n = mesh.n_vertices
        if getattr(u, "ndim", None) != 2 or tuple(u.shape) != (n, mesh.dim):
            raise ValueError("u must have shape [%d, %d]" % (n, mesh.dim))
        if _dtype_name(u) != "float64" or not _contiguous(u) or getattr(u, "is_cuda", False):
            raise ValueError("u must be contiguous float64 in host memory")
        if out is not None:
            for key, want, need in (("host", "int32", True), ("path_len", "int32", True),
                                    ("status", "uint8", True), ("start", "int32", False)):
                a = out.get(key)
                if a is None:
                    if need:
                        raise ValueError("out['%s'] is missing" % key)
                    continue
                if (_dtype_name(a) != want or not _contiguous(a) or _numel(a) < n
                        or getattr(a, "is_cuda", False)):
                    raise ValueError("out['%s'] must be contiguous %s in host memory with at "
                                     "least n = %d elements" % (key, want, n))
        if out is None:
            out = dict(host=np.empty(n, dtype=np.int32), path_len=np.empty(n, dtype=np.int32),
                       status=np.empty(n, dtype=np.uint8))
            if start_out:
                out["start"] = np.empty(n, dtype=np.int32)
        self._check(self.lib.cs_track_nodes_host(
            self.h, mesh.id, _field_id(field), _ptr(u), float(dt),
            MODES[mode] if isinstance(mode, str) else int(mode), _ptr(out["host"]),
            _ptr(out["path_len"]), _ptr(out["status"]), _ptr(out.get("start"))))
        return out

    def track_error(self, mesh, x, u, dt, host, start=None, dhat=None, stream=None):
        """Error statistics (Sec. 3.1) of a finished call: mean/max origin error
        err (centroid of the start element to centroid of the host) and, with
        a displacement grid dhat, mean/max |dhat * s - (x_p - x)|."""
        import torch
        check_track_args(mesh.dim, x, u, start)
        n = int(x.shape[0])
        if _dtype_name(host) != "int32" or not host.is_cuda or host.numel() < n:
            raise ValueError("host must be an int32 CUDA tensor of n elements")
        if dhat is not None:
            cells = int(np.prod(mesh.info()["pred_grid"]))
            if (_dtype_name(dhat) != "float32" or not dhat.is_cuda or not dhat.is_contiguous()
                    or dhat.numel() < cells * mesh.dim):
                raise ValueError("dhat must be a contiguous float32 CUDA tensor [%d, %d]"
                                 % (cells, mesh.dim))
        res = _capi.ErrorStats()
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        self._check(self.lib.cs_track_error(self.h, mesh.id, n, _ptr(x), _ptr(u), float(dt),
                                            _ptr(start), _ptr(host), _ptr(dhat),
                                            ctypes.byref(res), _stream_ptr(st)))
        return dict(n_err=res.n_err,
                    err_mean=res.err_sum / res.n_err if res.n_err else float("nan"),
                    err_max=res.err_max, n_disp=res.n_disp,
                    disp_mean=res.disp_sum / res.n_disp if res.n_disp else float("nan"),
                    disp_max=res.disp_max)

    # ---------------- start predictor ----------------
    def predictor_engine(self, engine):
        """'grid' (alias 'tc'): fully convolutional over the predictor grid on
        the tensor cores; 'tiles': the same pass on CUDA cores in 3-D;
        'window': every cell's own window through CUDA-core GEMMs."""
        code = {"tc": 1, "grid": 1, "tiles": 2, "window": 0}[engine]
        self._check(self.lib.cs_predictor_engine(self.h, code))

    def predictor_tile3(self, side=0):
        """Side of the 3-D tensor-core kernel's output tiles: 4, 3, 2 or 0
        (automatic)."""
        self._check(self.lib.cs_predictor_tile3(self.h, int(side)))

    def predictor_tile_rows(self, rows=0):
        """Tile height of the 2-D tensor-core grid kernel: 24, 13 or 8 rows,
        or 0 for the automatic choice."""
        self._check(self.lib.cs_predictor_tile_rows(self.h, int(rows)))

    def device_status(self):
        self._check(self.lib.cs_device_status(self.h))

    def debug_hold_predictor(self, on=True):
        """Test hook: the tensor-core predictor kernels first wait for a device
        flag that nothing sets, so that the wait runs out (CS_EDEVICE)."""
        self._check(self.lib.cs_debug_hold_predictor(self.h, 1 if on else 0))

    def predictor_precision(self, bf16=True):
        self._check(self.lib.cs_predictor_precision(self.h, 1 if bf16 else 0))

    def predictor_size(self, dim):
        return int(self.lib.cs_predictor_size(dim))

    def load_predictor(self, dim, weights):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self._check(self.lib.cs_predictor_load(self.h, dim, _ptr(w), w.size))

    def save_predictor(self, dim):
        out = np.empty(self.predictor_size(dim), dtype=np.float32)
        self._check(self.lib.cs_predictor_save(self.h, dim, _ptr(out), out.size))
        return out

    def grid_velocity(self, mesh, u_nodal, out=None, stream=None):
        """Resample the nodal velocity (float64 CUDA tensor) onto the ASG grid;
        out=None stores it in the mesh and returns None."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(u_nodal.device)
        self._check(self.lib.cs_grid_velocity(self.h, mesh.id, _ptr(u_nodal), _ptr(out),
                                              _stream_ptr(st)))
        return out

    def windows(self, mesh, dt, cells=None, B=None, grid=None, stream=None):
        import torch
        S = 9 if mesh.dim == 2 else 7
        B = cells.shape[0] if cells is not None else B
        out = torch.empty((B, mesh.dim) + (S,) * mesh.dim, dtype=torch.float32, device="cuda")
        st = stream if stream is not None else torch.cuda.current_stream()
        self._check(self.lib.cs_windows(self.h, mesh.id, _ptr(grid), float(dt), _ptr(cells), B,
                                        _ptr(out), _stream_ptr(st)))
        return out

    def predictor_forward(self, dim, windows):
        import torch
        out = torch.empty((windows.shape[0], dim), dtype=torch.float32, device=windows.device)
        self._check(self.lib.cs_predictor_forward(self.h, dim, windows.shape[0], _ptr(windows),
                                                  _ptr(out)))
        return out

    def predict(self, mesh, dt, out=None, stream=None):
        """Predicted displacement (cell units) at every ASG cell."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        self._check(self.lib.cs_predict(self.h, mesh.id, float(dt), _ptr(out), _stream_ptr(st)))
        return out

    def training_pairs(self, mesh, x, u, dt, stream=None):
        import torch
        n = x.shape[0]
        S = 9 if mesh.dim == 2 else 7
        win = torch.empty((n, mesh.dim) + (S,) * mesh.dim, dtype=torch.float32, device=x.device)
        tgt = torch.empty((n, mesh.dim), dtype=torch.float32, device=x.device)
        cells = torch.empty(n, dtype=torch.int64, device=x.device)
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        self._check(self.lib.cs_training_pairs(self.h, mesh.id, n, _ptr(x), _ptr(u), float(dt),
                                               _ptr(win), _ptr(tgt), _ptr(cells),
                                               _stream_ptr(st)))
        return win, tgt, cells

    def train(self, dim, windows, targets, batch=4096, steps=100, lr=1e-3, seed=0):
        losses = np.empty(steps, dtype=np.float32)
        self._check(self.lib.cs_predictor_train(self.h, dim, _ptr(windows), _ptr(targets),
                                                windows.shape[0], batch, steps, float(lr),
                                                int(seed), _ptr(losses)))
        return losses

    def predictor_grad(self, dim, windows, targets):
        import torch
        g = torch.empty(self.predictor_size(dim), dtype=torch.float32, device=windows.device)
        loss = np.zeros(1, dtype=np.float32)
        self._check(self.lib.cs_predictor_grad(self.h, dim, windows.shape[0], _ptr(windows),
                                               _ptr(targets), _ptr(g), _ptr(loss)))
        return g, float(loss[0])

    def track_dhat(self, mesh, x, u, dt, dhat=None, start=None, out=None, start_out=False,
                   stream=None):
        """CNN-SNS start rule with a given displacement grid dhat (float32 CUDA
        [prod pred_grid, dim], predictor cell units; None = the mesh's stored
        prediction)."""
        import torch
        n = check_track_args(mesh.dim, x, u, start, out)
        if dhat is not None:
            cells = int(np.prod(mesh.info()["pred_grid"]))
            if (_dtype_name(dhat) != "float32" or not dhat.is_cuda or not dhat.is_contiguous()
                    or dhat.numel() < cells * mesh.dim):
                raise ValueError("dhat must be a contiguous float32 CUDA tensor [%d, %d]"
                                 % (cells, mesh.dim))
        out = self._device_out(n, x.device, out, start_out)
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        self._check(self.lib.cs_track_dhat(
            self.h, mesh.id, n, _ptr(x), _ptr(u), float(dt), _ptr(start), _ptr(dhat),
            _ptr(out["host"]), _ptr(out["path_len"]), _ptr(out["status"]),
            _ptr(out.get("start")), _stream_ptr(st)))
        return out

    # ---------------- classifier predictor (Sec. 2.3, Eq. 7-8) ----------------
    def classifier_size(self, dim):
        return int(self.lib.cs_classifier_size(dim))

    def classifier_window(self, dim):
        return int(self.lib.cs_classifier_window(dim))

    def load_classifier(self, dim, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.classifier_size(dim):
            raise ValueError("the classifier of dim %d has %d parameters, not %d"
                             % (dim, self.classifier_size(dim), p.size))
        self._check(self.lib.cs_classifier_load(self.h, dim, _ptr(p), p.size))

    def save_classifier(self, dim):
        out = np.empty(self.classifier_size(dim), dtype=np.float32)
        self._check(self.lib.cs_classifier_save(self.h, dim, _ptr(out), out.size))
        return out

    def _xp_rows(self, mesh, xp, name="xp"):
        _check_dev(name, xp, "float64", (None, mesh.dim))
        return int(xp.shape[0])

    def departure(self, mesh, x, u, dt, stream=None):
        """x_p = x - (u * dt) on the device (float64 CUDA [n, dim])."""
        import torch
        n = check_track_args(mesh.dim, x, u)
        xp = torch.empty((n, mesh.dim), dtype=torch.float64, device=x.device)
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        self._check(self.lib.cs_departure(self.h, mesh.id, n, _ptr(x), _ptr(u), float(dt),
                                          _ptr(xp), _stream_ptr(st)))
        return xp

    def classifier_features(self, mesh, xp, stream=None):
        """(window [n, dim, W..W], offset [n, dim]) float32 CUDA tensors."""
        import torch
        n = self._xp_rows(mesh, xp)
        W = self.classifier_window(mesh.dim)
        win = torch.empty((n, mesh.dim) + (W,) * mesh.dim, dtype=torch.float32, device=xp.device)
        off = torch.empty((n, mesh.dim), dtype=torch.float32, device=xp.device)
        st = stream if stream is not None else torch.cuda.current_stream(xp.device)
        self._check(self.lib.cs_classifier_features(self.h, mesh.id, n, _ptr(xp), _ptr(win),
                                                    _ptr(off), _stream_ptr(st)))
        return win, off

    def classifier_forward(self, mesh, xp):
        """Logits [n, W^dim] (float32 CUDA) of departure points xp."""
        import torch
        n = self._xp_rows(mesh, xp)
        ncls = self.classifier_window(mesh.dim) ** mesh.dim
        out = torch.empty((n, ncls), dtype=torch.float32, device=xp.device)
        torch.cuda.current_stream(xp.device).synchronize()
        self._check(self.lib.cs_classifier_forward(self.h, mesh.id, n, _ptr(xp), _ptr(out)))
        return out

    def classifier_labels(self, mesh, xp, host, stream=None):
        import torch
        n = self._xp_rows(mesh, xp)
        _check_dev("host", host, "int32", (n,), xp.device)
        out = torch.empty(n, dtype=torch.int32, device=xp.device)
        st = stream if stream is not None else torch.cuda.current_stream(xp.device)
        self._check(self.lib.cs_classifier_labels(self.h, mesh.id, n, _ptr(xp), _ptr(host),
                                                  _ptr(out), _stream_ptr(st)))
        return out

    def classifier_pairs(self, mesh, x, u, dt, start=None, stream=None):
        """(xp [n, dim] float64, labels [n] int32) CUDA tensors by plain SNS."""
        import torch
        n = check_track_args(mesh.dim, x, u, start)
        xp = torch.empty((n, mesh.dim), dtype=torch.float64, device=x.device)
        lab = torch.empty(n, dtype=torch.int32, device=x.device)
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        self._check(self.lib.cs_classifier_pairs(self.h, mesh.id, n, _ptr(x), _ptr(u), float(dt),
                                                 _ptr(start), _ptr(xp), _ptr(lab),
                                                 _stream_ptr(st)))
        return xp, lab

    def classifier_grad(self, mesh, xp, labels):
        import torch
        n = self._xp_rows(mesh, xp)
        _check_dev("labels", labels, "int32", (n,), xp.device)
        g = torch.empty(self.classifier_size(mesh.dim), dtype=torch.float32, device=xp.device)
        loss = np.zeros(1, dtype=np.float32)
        torch.cuda.current_stream(xp.device).synchronize()
        self._check(self.lib.cs_classifier_grad(self.h, mesh.id, n, _ptr(xp), _ptr(labels),
                                                _ptr(g), _ptr(loss)))
        return g, float(loss[0])

    def train_classifier(self, mesh, xp, labels, batch=4096, steps=100, lr=1e-3, seed=0):
        import torch
        n = self._xp_rows(mesh, xp)
        _check_dev("labels", labels, "int32", (n,), xp.device)
        losses = np.empty(steps, dtype=np.float32)
        torch.cuda.current_stream(xp.device).synchronize()
        self._check(self.lib.cs_classifier_train(self.h, mesh.id, _ptr(xp), _ptr(labels), n,
                                                 int(batch), int(steps), float(lr), int(seed),
                                                 _ptr(losses)))
        return losses

    def classifier_start(self, mesh, xp, logits, fallback=None, stream=None):
        """(start [n] user ids, class [n]) int32 CUDA tensors from logits."""
        import torch
        n = self._xp_rows(mesh, xp)
        _check_dev("logits", logits, "float32",
                   (n, self.classifier_window(mesh.dim) ** mesh.dim), xp.device)
        if fallback is not None:
            _check_dev("fallback", fallback, "int32", (n,), xp.device)
        elif n != mesh.n_vertices:
            raise ValueError("fallback is needed unless the particles are the mesh nodes")
        start = torch.empty(n, dtype=torch.int32, device=xp.device)
        cls = torch.empty(n, dtype=torch.int32, device=xp.device)
        st = stream if stream is not None else torch.cuda.current_stream(xp.device)
        self._check(self.lib.cs_classifier_start(self.h, mesh.id, n, _ptr(xp), _ptr(logits),
                                                 _ptr(fallback), _ptr(start), _ptr(cls),
                                                 _stream_ptr(st)))
        return start, cls

    def track_classifier(self, mesh, x, u, dt, start=None, out=None, start_out=False,
                         stream=None):
        """CNN-SNS with the classifier's start (Eq. 8); same arrays as track()."""
        import torch
        n = check_track_args(mesh.dim, x, u, start, out)
        out = self._device_out(n, x.device, out, start_out)
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        self._check(self.lib.cs_track_classifier(
            self.h, mesh.id, n, _ptr(x), _ptr(u), float(dt), _ptr(start), _ptr(out["host"]),
            _ptr(out["path_len"]), _ptr(out["status"]), _ptr(out.get("start")),
            _stream_ptr(st)))
        return out

    # ---------------- serving ----------------
    def serve_start(self, slots=4, arena_bytes=2 << 30):
        cfg = _capi.ServeCfg(slots, arena_bytes)
        self._check(self.lib.cs_serve_start(self.h, ctypes.byref(cfg)))
        self._requests = {}

    def submit(self, mesh, x, u, dt, start=None, mode="sns", field=None, out=None):
        """Queue a request (host arrays, pinned torch tensors overlap best).
        out: the caller's host arrays host, path_len (int32) and status
        (uint8) of at least n elements (a server reuses its pinned result
        buffers), else new pinned ones. Returns (ticket, outputs); outputs are
        valid after wait(ticket)."""
        import torch
        if out is not None and any(out.get(k) is None for k in ("host", "path_len", "status")):
            raise ValueError("out needs host, path_len and status")
        n = check_track_args(mesh.dim, x, u, start, out=out, on_device=False)
        if out is None:
            out = dict(host=torch.empty(n, dtype=torch.int32, pin_memory=True),
                       path_len=torch.empty(n, dtype=torch.int32, pin_memory=True),
                       status=torch.empty(n, dtype=torch.uint8, pin_memory=True))
        req = _capi.Request(mesh.id, _field_id(field), n, _ptr(x), _ptr(u), float(dt),
                            _ptr(start),
                            MODES[mode] if isinstance(mode, str) else int(mode),
                            _ptr(out["host"]), _ptr(out["path_len"]), _ptr(out["status"]))
        t = ctypes.c_int64()
        self._check(self.lib.cs_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        self._requests[t.value] = (x, u, start, out)   # keep the arrays alive
        return t.value, out

    def wait(self, ticket, timeout_ms=60000):
        """Block until the request finishes; returns the start rule it ran with."""
        res, mode = ctypes.c_int32(), ctypes.c_int32()
        rc = self.lib.cs_serve_wait(self.h, ticket, int(timeout_ms), ctypes.byref(res),
                                    ctypes.byref(mode))
        if rc == -4:
            raise TimeoutError("request %d still running" % ticket)
        self._check(rc)
        self._check(res.value)
        self._requests.pop(ticket, None)
        return mode.value

    def serve_report(self):
        s = _capi.ServeStats()
        self._check(self.lib.cs_serve_report(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _capi.ServeStats._fields_}

    def serve_trace(self):
        """Records of the requests finished so far, in finishing order: dicts
        of ticket, n, mesh_id, mode_used, slot, in_flight, result, dt, the
        submit, admit and done times in ms since the first submit, and the
        device times of the request's stages (h2d_ms, predict_ms, walk_ms,
        d2h_ms)."""
        count = ctypes.c_int64()
        self._check(self.lib.cs_serve_trace(self.h, 0, None, ctypes.byref(count)))
        recs = (_capi.ServeRecord * max(count.value, 1))()
        self._check(self.lib.cs_serve_trace(self.h, count.value, recs, ctypes.byref(count)))
        return [{k: getattr(recs[i], k) for k, _ in _capi.ServeRecord._fields_ if k != "reserved"}
                for i in range(count.value)]

    def serve_stop(self):
        self._check(self.lib.cs_serve_stop(self.h))

    def stats(self, path_len, status, stream=None):
        """(sum, max, count FOUND, OUTSIDE, FALLBACK, INVALID) of device outputs."""
        import torch
        res = (ctypes.c_int64 * 6)()
        st = stream if stream is not None else torch.cuda.current_stream(path_len.device)
        self._check(self.lib.cs_track_stats(self.h, path_len.shape[0], _ptr(path_len),
                                            _ptr(status), res, _stream_ptr(st)))
        return dict(sum=res[0], max=res[1], found=res[2], outside=res[3], fallback=res[4],
                    invalid=res[5])
