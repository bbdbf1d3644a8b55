"""The Python binding refuses malformed arrays before any pointer reaches the
C ABI (CPU only). The library trusts the sizes it is given, so a float32,
non-contiguous, wrong-width or short array would make a kernel read or write
past it; the binding must raise ValueError and call nothing."""

import numpy as np
import pytest
import torch

import paper_2412_18379_gb300 as cs
from paper_2412_18379_gb300 import check_track_args


class _NoCalls:
    """Stands in for the loaded library: any attribute access is a failure."""

    def __getattr__(self, name):
        raise AssertionError("the binding called %s" % name)


class _FakeMesh:
    def __init__(self, dim, n_v=10):
        self.id = 1
        self.dim = dim
        self.n_vertices = n_v
        self.n_elements = 2 * n_v


def _ctx():
    ctx = object.__new__(cs.Context)
    ctx.lib = _NoCalls()
    ctx.h = None
    return ctx


def _good(n=8, dim=2):
    return (torch.zeros((n, dim), dtype=torch.float64), torch.zeros((n, dim), dtype=torch.float64),
            torch.zeros(n, dtype=torch.int32))


def test_accepts_well_formed_host_arrays():
    x, u, s = _good()
    out = dict(host=np.empty(8, np.int32), path_len=np.empty(8, np.int32),
               status=np.empty(8, np.uint8), start=np.empty(8, np.int32))
    assert check_track_args(2, x, u, s, out, on_device=False) == 8
    assert check_track_args(3, np.zeros((5, 3)), np.zeros((5, 3)), on_device=False) == 5


@pytest.mark.parametrize("bad", ["x_f32", "u_f32", "x_dim", "u_rows", "x_strided",
                                 "start_i64", "start_len", "out_short", "status_i32",
                                 "host_f32"])
def test_rejects_malformed_arrays(bad):
    x, u, s = _good()
    out = dict(host=np.empty(8, np.int32), path_len=np.empty(8, np.int32),
               status=np.empty(8, np.uint8))
    if bad == "x_f32":
        x = x.float()
    elif bad == "u_f32":
        u = u.float()
    elif bad == "x_dim":
        x = torch.zeros((8, 3), dtype=torch.float64)
    elif bad == "u_rows":
        u = torch.zeros((7, 2), dtype=torch.float64)
    elif bad == "x_strided":
        x = torch.zeros((2, 8), dtype=torch.float64).t()
    elif bad == "start_i64":
        s = s.long()
    elif bad == "start_len":
        s = torch.zeros(7, dtype=torch.int32)
    elif bad == "out_short":
        out["path_len"] = np.empty(7, np.int32)
    elif bad == "status_i32":
        out["status"] = np.empty(8, np.int32)
    elif bad == "host_f32":
        out["host"] = np.empty(8, np.float32)
    with pytest.raises(ValueError):
        check_track_args(2, x, u, s, out, on_device=False)


def test_device_calls_need_cuda_tensors():
    x, u, s = _good()
    with pytest.raises(ValueError):
        check_track_args(2, x, u, s, on_device=True)


@pytest.mark.parametrize("call", ["track", "track_noalloc", "track_dhat", "track_host",
                                  "track_classifier", "classifier_pairs", "departure"])
def test_entry_points_raise_before_calling_the_library(call):
    ctx = _ctx()
    mesh = _FakeMesh(2)
    x = torch.zeros((8, 2), dtype=torch.float32)        # wrong dtype
    u = torch.zeros((8, 2), dtype=torch.float64)
    with pytest.raises(ValueError):
        getattr(ctx, call)(mesh, x, u, 0.1)
    x = torch.zeros((8, 3), dtype=torch.float64)        # wrong width for a 2-D mesh
    with pytest.raises(ValueError):
        getattr(ctx, call)(mesh, x, torch.zeros((8, 3), dtype=torch.float64), 0.1)


def test_field_upload_checks_shape_before_calling_the_library():
    ctx = _ctx()
    mesh = _FakeMesh(2, n_v=10)
    with pytest.raises(ValueError):
        ctx.upload_field(mesh, np.zeros((9, 2)))
    with pytest.raises(ValueError):
        ctx.upload_field(mesh, torch.zeros((10, 2), dtype=torch.float32))


@pytest.mark.parametrize("call", ["classifier_features", "classifier_forward"])
def test_classifier_calls_check_the_points_first(call):
    """The classifier's entry points take float64 CUDA departure points of the
    mesh's width; anything else is refused before the library is called."""
    ctx = _ctx()
    mesh = _FakeMesh(2)
    for xp in (torch.zeros((8, 2), dtype=torch.float64),               # host memory
               torch.zeros((8, 2), dtype=torch.float32),               # wrong dtype
               torch.zeros((8, 3), dtype=torch.float64),               # wrong width
               torch.zeros((2, 8), dtype=torch.float64).t()):          # strided
        with pytest.raises(ValueError):
            getattr(ctx, call)(mesh, xp)


def test_classifier_parameters_are_sized_before_the_library_is_called():
    ctx = _ctx()
    ctx.classifier_size = lambda dim: 100
    with pytest.raises(ValueError):
        ctx.load_classifier(2, np.zeros(99, dtype=np.float32))


def test_submit_checks_the_callers_result_buffers():
    """A served request writes its results into the caller's buffers when
    given: short, mistyped, incomplete or device buffers are refused before
    the library is called."""
    ctx = _ctx()
    mesh = _FakeMesh(2)
    x, u, s = _good()
    good = dict(host=np.empty(8, np.int32), path_len=np.empty(8, np.int32),
                status=np.empty(8, np.uint8))
    bad = [dict(good, host=np.empty(7, np.int32)),
           dict(good, status=np.empty(8, np.int32)),
           {k: v for k, v in good.items() if k != "path_len"}]
    if torch.cuda.is_available():
        bad.append(dict(good, host=torch.empty(8, dtype=torch.int32, device="cuda")))
    for out in bad:
        with pytest.raises(ValueError):
            ctx.submit(mesh, x, u, 0.1, start=s, mode="sns", out=out)


def test_nodes_call_checks_the_velocity_first():
    """cs_track_nodes_host reads u [n_v, dim] float64 from host memory; a
    wrong shape, dtype or layout is refused before the library is called."""
    ctx = _ctx()
    mesh = _FakeMesh(2, n_v=10)
    for u in (np.zeros((9, 2)), np.zeros((10, 3)), torch.zeros((10, 2), dtype=torch.float32),
              torch.zeros((2, 10), dtype=torch.float64).t()):
        with pytest.raises(ValueError):
            ctx.track_nodes_host(mesh, u, 0.1)
    with pytest.raises(ValueError):
        ctx.track_nodes_host(mesh, np.zeros((10, 2)), 0.1,
                             out=dict(host=np.empty(9, np.int32), path_len=np.empty(10, np.int32),
                                      status=np.empty(10, np.uint8)))


def test_nodes_call_passes_its_arguments_through():
    """A well-formed call reaches cs_track_nodes_host once, with the mesh and
    field ids, u's address, dt, the mode and the output addresses as given."""
    calls = []

    class _Record:
        def __getattr__(self, name):
            def f(*args):
                calls.append((name, args))
                return 0
            return f

    ctx = object.__new__(cs.Context)
    ctx.lib = _Record()
    ctx.h = None
    mesh = _FakeMesh(2, n_v=10)
    u = torch.zeros((10, 2), dtype=torch.float64)
    out = dict(host=np.empty(10, np.int32), path_len=np.empty(10, np.int32),
               status=np.empty(10, np.uint8))
    got = ctx.track_nodes_host(mesh, u, 0.25, mode="cnn", out=out, field=7)
    assert got is out
    assert [c[0] for c in calls] == ["cs_track_nodes_host"]
    args = calls[0][1]
    assert args[1:6] == (mesh.id, 7, u.data_ptr(), 0.25, cs.CS_CNN_SNS)
    assert args[6:] == (out["host"].ctypes.data, out["path_len"].ctypes.data,
                        out["status"].ctypes.data, None)
