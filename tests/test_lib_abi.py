"""CPU-side checks of the C ABI: the library loads, exports every entry point declared in
include/mf.h, and validates arguments on the host (no GPU compute is called here)."""
import ctypes as C
import os
import re

import pytest

import paper_2609_04534_gb300 as mf
from paper_2609_04534_gb300 import build as mfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    mfbuild.build()
    return mf.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mf_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "mf_apply" in names and "mf_cg_solve" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_mesh_argument_validation(L):
    with pytest.raises(mf.MfError) as e:
        mf.mf_mesh_create(0, 4, 4)
    assert e.value.code == mf.MF_ERR_ARG
    with pytest.raises(mf.MfError):
        mf.mf_mesh_create(4, 4, 4, 7)
    with pytest.raises(mf.MfError):
        mf.mf_mesh_create(4, 4, 4, mf.MF_CURVED_SIN, None, 0.5)  # would fold the mesh
    m = mf.mf_mesh_create(4, 4, 4, mf.MF_CURVED_SIN, None, 0.1)
    mf.mf_mesh_destroy(m)


def test_operator_argument_validation_and_info(L):
    m = mf.mf_mesh_create(5, 6, 3)
    for bad in [dict(degree=0), dict(degree=9), dict(degree=2, kind=5), dict(degree=2, precision=9),
                dict(degree=2, bc=3)]:
        kw = dict(kind=mf.MF_LAPLACE, precision=mf.MF_FP64, bc=mf.MF_BC_NONE)
        kw.update(bad)
        with pytest.raises(mf.MfError) as e:
            mf.mf_operator_create(m, kw.pop("degree"), **kw)
        assert e.value.code == mf.MF_ERR_ARG
    op = mf.mf_operator_create(m, 3)
    info = mf.mf_operator_info(op)
    assert info["n_cellwise"] == 5 * 6 * 3 * 64
    assert info["n_unique"] == 16 * 19 * 10
    # tiles of 4x4x2 cells: ceil(5/4)*ceil(6/4)*ceil(3/2) = 2*2*2 tiles of 32 lanes
    assert info["n_native"] == 8 * 32 * 64
    assert info["path"] == 0 and info["geom_bytes"] == 0
    assert info["algorithmic_bytes_per_apply"] == 16 * info["n_cellwise"]
    mf.mf_operator_destroy(op)
    mc = mf.mf_mesh_create(5, 6, 3, mf.MF_CURVED_SIN, None, 0.1)
    op = mf.mf_operator_create(mc, 4, mf.MF_HELMHOLTZ, 1.0, mf.MF_MIXED, mf.MF_BC_DIRICHLET0)
    info = mf.mf_operator_info(op)
    assert info["path"] == 2
    # FP64 view streams 7 values per point; the FP32 view keeps sin/cos tables per cell layer
    assert info["geom_bytes"] == 7 * info["n_native"] * 8 + 4 * 2 * (5 + 6 + 3) * 5
    assert info["algorithmic_bytes_per_apply"] == (16 + 7 * 8) * info["n_cellwise"]
    # not set up yet: apply and its stream twin must refuse without touching the GPU
    for fn in (mf.mf_apply, mf.mf_apply_stream_twin):
        with pytest.raises(mf.MfError) as e:
            fn(op, 16, 32)
        assert e.value.code == mf.MF_ERR_ARG
    # workspace too small
    with pytest.raises(mf.MfError) as e:
        mf.mf_operator_setup(op, 256, 1024)
    assert e.value.code == mf.MF_ERR_OOM
    assert mf.mf_cg_workspace_bytes(op, 1) > mf.mf_cg_workspace_bytes(op, 0) > 0
    # solver entry points refuse before touching the GPU: bad CG form, operator not set up
    with pytest.raises(mf.MfError) as e:
        mf.mf_cg_solve(op, 16, 32, 1e-10, 10, 0, 256, 1 << 30, cg_form=7)
    assert e.value.code == mf.MF_ERR_ARG
    with pytest.raises(mf.MfError) as e:  # Jacobi needs the split-dual form
        mf.mf_cg_solve(op, 16, 32, 1e-10, 10, 0, 256, 1 << 30, cg_form=mf.MF_CG_ASSEMBLED,
                       precond=mf.MF_PRECOND_JACOBI)
    assert e.value.code == mf.MF_ERR_ARG
    for its, form in [(10, 0), (0, 1), (1001, 1), (5, 4)]:
        with pytest.raises(mf.MfError) as e:
            mf.mf_cg_profile(op, 16, 32, its, form, 256, 1 << 30)
        assert e.value.code == mf.MF_ERR_ARG
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mc)
    mf.mf_mesh_destroy(m)


def test_stream_twin_argument_validation(L):
    with pytest.raises(mf.MfError) as e:
        mf.mf_apply_stream_twin(None, 16, 32)
    assert e.value.code == mf.MF_ERR_ARG
    assert "NULL operator" in mf.last_error()


def test_noalloc_dot_rejects_on_the_host(L):
    """mf_dot_noalloc refuses on the host, before any CUDA call: a vector longer than its
    static scratch (134,217,728 native elements), then an operator that was never set up.
    The pointers are never dereferenced: no operator here is set up, so even a regressed
    size check stops at the set-up check."""
    mesh = mf.mf_mesh_create(256, 256, 128)
    op = mf.mf_operator_create(mesh, 3)
    assert mf.mf_operator_info(op)["n_native"] > 134_217_728
    with pytest.raises(mf.MfError) as e:
        mf.mf_dot_noalloc(op, 256, 512, 1024)
    assert e.value.code == mf.MF_ERR_ARG
    assert "limit" in str(e.value)
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)
    mesh = mf.mf_mesh_create(4, 4, 4)
    op = mf.mf_operator_create(mesh, 3)
    with pytest.raises(mf.MfError) as e:
        mf.mf_dot_noalloc(op, 256, 512, 1024)
    assert e.value.code == mf.MF_ERR_ARG
    assert "not set up" in str(e.value)
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)


def test_cg_solve_host_argument_validation(L):
    mesh = mf.mf_mesh_create(4, 4, 4)
    op = mf.mf_operator_create(mesh, 2)
    with pytest.raises(mf.MfError) as e:
        mf.mf_cg_solve_host(op, 16, 32, 1e-8, 10, 0, 256, 1 << 20)
    assert e.value.code == mf.MF_ERR_ARG and "not set up" in str(e.value)
    with pytest.raises(mf.MfError) as e:
        mf.mf_cg_solve_host(None, 16, 32, 1e-8, 10, 0, 256, 1 << 20)
    assert e.value.code == mf.MF_ERR_ARG
    assert mf.mf_cg_solve_host_workspace_bytes(op, 0) > mf.mf_cg_workspace_bytes(op, 0)
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)


def test_make_consistent_argument_validation(L):
    with pytest.raises(mf.MfError) as e:
        mf.mf_make_consistent(None, 16)
    assert e.value.code == mf.MF_ERR_ARG


def test_sheared_affine_selects_general_path(L):
    m = mf.mf_mesh_create(2, 2, 2, mf.MF_AFFINE, [1, 0.3, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0])
    op = mf.mf_operator_create(m, 2)
    assert mf.mf_operator_info(op)["path"] == 1
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(m)
    m = mf.mf_mesh_create(2, 2, 2, mf.MF_AFFINE, [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0])
    with pytest.raises(mf.MfError):
        mf.mf_operator_create(m, 2)
    mf.mf_mesh_destroy(m)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(mf, "_lib", None)
    monkeypatch.setattr(mf, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        mf.lib()


def test_mixed_restart_option_validation(L):
    """The mixed solver's restart switch and the server's copy of it accept 0 or 1 only; the
    checks run before any device call."""
    mesh = mf.mf_mesh_create(4, 4, 4)
    op = mf.mf_operator_create(mesh, 2)
    for bad in (-1, 2):
        with pytest.raises(mf.MfError) as e:
            mf.mf_cg_solve(op, 256, 512, 1e-8, 10, 1, 256, 1 << 20, mixed_restart=bad)
        assert e.value.code == mf.MF_ERR_ARG and "bad options" in str(e.value)
        with pytest.raises(mf.MfError) as e:
            mf.mf_server_create(256, 1 << 20, mixed_restart=bad)
        assert e.value.code == mf.MF_ERR_ARG and "mixed_restart" in str(e.value)
    with pytest.raises(mf.MfError) as e:
        mf.mf_server_create(256, 1 << 20, inner_rtol=1.5)
    assert e.value.code == mf.MF_ERR_ARG
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)


def test_block_sweep_argument_validation(L):
    """mf_apply_split_block checks B before the operator's state (not set up: MF_ERR_ARG)."""
    mesh = mf.mf_mesh_create(4, 4, 4)
    for k, b, code in ((3, 5, mf.MF_ERR_ARG), (3, 64, mf.MF_ERR_ARG), (2, 8, mf.MF_ERR_ARG),
                       (3, 8, mf.MF_ERR_ARG)):
        op = mf.mf_operator_create(mesh, k)
        with pytest.raises(mf.MfError) as e:
            mf.mf_apply_split_block(op, b, 256, 512)
        assert e.value.code == code, (k, b)
        mf.mf_operator_destroy(op)
    with pytest.raises(mf.MfError) as e:
        mf.mf_apply_split_block(None, 8, 256, 512)
    assert e.value.code == mf.MF_ERR_ARG
    mf.mf_mesh_destroy(mesh)
