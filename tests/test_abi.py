"""The C-ABI library loads, exports every symbol include/trsgd.h declares, and
rejects malformed arguments on the host before any CUDA call (CPU only)."""
import ctypes

import pytest

from paper_2303_16492_gb300 import _abi
from paper_2303_16492_gb300 import build as _build


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _abi.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _abi.header_symbols()
    assert "trsgd_init" in names and "trsgd_step" in names and "trsgd_run" in names
    assert "trsgd_rel_error" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []
    assert set(names) == set(_abi._SIGNATURES)


def test_debug_build_exports_every_symbol():
    """The debug build (index checks compiled in) links and exports the same
    entry points; loaded on its own, without touching the product library."""
    import ctypes as C
    path = _build.build(debug=True)
    L = C.CDLL(path)
    assert [n for n in _abi.header_symbols() if not hasattr(L, n)] == []
    L.trsgd_status_string.restype = C.c_char_p
    assert b"index" in L.trsgd_status_string(_abi.EBADINDEX)


def test_status_strings(lib):
    for s in range(8):
        assert _abi.status_string(s) != "unknown status"
    assert "invalid" in _abi.status_string(_abi.EINVAL)
    assert "index" in _abi.status_string(_abi.EBADINDEX)


def test_config_struct_layout():
    assert ctypes.sizeof(_abi.Config) == 224
    assert _abi.Config.I.offset == 8 and _abi.Config.seed.offset == 208 and _abi.Config.path.offset == 216


def _cfg(**kw):
    c = _abi.Config()
    c.N = 3
    for k in range(3):
        c.I[k] = 10
        c.R[k] = 2
    c.J = 8
    c.prec = _abi.FP32
    c.x_dtype = _abi.DTYPE_F32
    c.alpha = 0.1
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _init(lib, cfg, n=1, xs=True, cores=True):
    arr = (_abi.Config * n)(*([cfg] * n))
    X = (ctypes.c_void_p * n)(*([ctypes.c_void_p(0x1000)] * n)) if xs else None
    C = (ctypes.c_void_p * (3 * n))(*([ctypes.c_void_p(0x2000)] * (3 * n))) if cores else None
    h = ctypes.c_void_p()
    return lib.trsgd_init(arr, n, X, C, None, ctypes.byref(h)), h


@pytest.mark.parametrize("field,value", [
    ("N", 1), ("N", 9), ("J", 0), ("J_H", -1), ("dist", 7), ("variant", 2), ("rule", -1),
    ("prec", 5), ("x_dtype", 3), ("alpha", float("nan")), ("damping", -1.0), ("eta", -0.5),
])
def test_invalid_config_rejected_on_host(lib, field, value):
    st, h = _init(lib, _cfg(**{field: value}))
    assert st == _abi.EINVAL and not h.value


def test_invalid_dims_and_ranks(lib):
    c = _cfg()
    c.I[1] = 0
    assert _init(lib, c)[0] == _abi.EINVAL
    c = _cfg()
    c.R[2] = 0
    assert _init(lib, c)[0] == _abi.EINVAL


def test_precision_dtype_mismatch(lib):
    assert _init(lib, _cfg(prec=_abi.FP64, x_dtype=_abi.DTYPE_F32))[0] == _abi.EINVAL
    assert _init(lib, _cfg(prec=_abi.FP32, x_dtype=_abi.DTYPE_F64))[0] == _abi.EINVAL


def test_null_pointers(lib):
    assert _init(lib, _cfg(), xs=False)[0] == _abi.EINVAL
    assert _init(lib, _cfg(), cores=False)[0] == _abi.EINVAL
    arr = (_abi.Config * 1)(_cfg())
    assert lib.trsgd_init(arr, 1, None, None, None, None) == _abi.EINVAL
    assert lib.trsgd_init(None, 1, None, None, None, ctypes.byref(ctypes.c_void_p())) == _abi.EINVAL
    assert lib.trsgd_init(arr, 0, None, None, None, ctypes.byref(ctypes.c_void_p())) == _abi.EINVAL


def test_unsupported_shapes_reported(lib):
    c = _cfg(path=_abi.PATH_CLUSTER)
    c.R[0] = 17                          # rank beyond the fused kernel's registers
    assert _init(lib, c)[0] == _abi.EUNSUPPORTED
    c = _cfg()
    c.R[0] = 33                          # beyond both paths
    assert _init(lib, c)[0] == _abi.EUNSUPPORTED
    c = _cfg(dist=_abi.DIST_EUCLIDEAN)
    c.R[0] = 17                          # the whole-GPU path samples uniformly only
    assert _init(lib, c)[0] == _abi.EUNSUPPORTED
    c = _cfg(variant=_abi.SCALED)
    for k in range(3):
        c.R[k] = 23                      # Q = 529 > the scaled limits of both paths (128, 512)
    assert _init(lib, c)[0] == _abi.EUNSUPPORTED
    c = _cfg(variant=_abi.SCALED, prec=_abi.FP64, x_dtype=_abi.DTYPE_F64)
    for k in range(3):
        c.R[k] = 12                      # Q = 144: the whole-GPU path has no FP64 mode
    assert _init(lib, c)[0] == _abi.EUNSUPPORTED
    c = _cfg(path=_abi.PATH_GRID, prec=_abi.FP64, x_dtype=_abi.DTYPE_F64)
    assert _init(lib, c)[0] == _abi.EUNSUPPORTED


def test_path_field_validated(lib):
    assert _init(lib, _cfg(path=3))[0] == _abi.EINVAL
    assert _init(lib, _cfg(fp32_units=2))[0] == _abi.EINVAL
    # the whole-GPU path runs FP32 on tensor-core pieces only
    assert _init(lib, _cfg(path=_abi.PATH_GRID, fp32_units=_abi.FP32_FMA))[0] == _abi.EUNSUPPORTED


def test_null_handle_calls(lib):
    assert lib.trsgd_step(None, 0) == _abi.EINVAL
    assert lib.trsgd_run(None, 0, 1, 0, 0.0, 0.0, None, None, None) == _abi.EINVAL
    out = ctypes.c_double()
    assert lib.trsgd_rel_error(None, 0, None, ctypes.byref(out)) == _abi.EINVAL
    assert lib.trsgd_set_debug(None, 1) == _abi.EINVAL
    assert lib.trsgd_debug_index_bound(None, 0, 0) == _abi.EINVAL
    assert lib.trsgd_launch_count(None) == -1
    assert lib.trsgd_tensor_pieces(None) == -1
    assert lib.trsgd_gd_step(None, 0, 0.1, 0.0) == _abi.EINVAL
    sh = _abi.Shard()
    assert lib.trsgd_shard_plan(None, 0, 0, 1, ctypes.byref(sh)) == _abi.EINVAL
    assert lib.trsgd_step_partial(None, 0, ctypes.byref(sh), ctypes.c_void_p(16), None) == _abi.EINVAL
    assert lib.trsgd_step_apply(None, 0, ctypes.c_void_p(16), 1, None, 0) == _abi.EINVAL
    lib.trsgd_destroy(None)


def test_reconstruct_and_adjoint_validate_on_host(lib):
    I = (ctypes.c_int64 * 3)(4, 4, 4)
    R = (ctypes.c_int64 * 3)(2, 2, 2)
    assert lib.trsgd_reconstruct(1, I, R, 1, None, None, None) == _abi.EINVAL
    assert lib.trsgd_reconstruct(3, I, R, 1, None, ctypes.c_void_p(16), None) == _abi.EINVAL
    assert lib.trsgd_sampled_loss_grad(3, I, R, 3, 4, None, None, None, None, None, None, None) == _abi.EINVAL
