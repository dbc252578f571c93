"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point declared in include/*.h, and rejects bad arguments on the host
(no compute calls are made here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(fwi_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1406_1864_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["fwi_forward", "fwi_adjoint_gradient", "fwi_illumination", "fwi_offset_hessian_diag",
                 "fwi_adjoint_apply", "fwi_workspace_bytes", "fwi_last_error", "fwi_batch_gradient",
                 "fwi_batch_workspace_bytes", "fwi_exec_gradient_create", "fwi_exec_run", "fwi_exec_destroy",
                 "fwi_autotune", "fwi_autotune_reset", "fwi_autotune_set", "fwi_born",
                 "fwi_gauss_newton_hvp", "fwi_misfit", "fwi_receiver_factor", "fwi_precondition_receiver",
                 "fwi_extended_born", "fwi_extended_migration", "fwi_exec_input_ready",
                 "fwi_plessix_mulder_hessian", "fwi_selftest_wait"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert lib.fwi_version() >= 100


def test_library_is_sm103a_only():
    from paper_1406_1864_gb300 import build as b
    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)


def _structs(nz=30, nx=40, nt=100, ns=2, nrec=5):
    from paper_1406_1864_gb300 import _lib as L
    g = L.FwiGrid(2, nz, 1, nx, 10.0, 1e-3, nt, 10, 3000.0, 0.05)
    src = np.zeros((ns, 3), np.int32)
    src[:, 2] = [5, 30][:ns] if ns <= 2 else np.arange(ns) % nx
    rec = np.zeros((ns, nrec, 3), np.int32)
    rec[:, :, 2] = np.arange(nrec)
    ge = L.FwiGeometry(ns, nrec, src.ctypes.data, rec.ctypes.data, 1)
    o = L.FwiOptions(0, 0, 3, 1, 1e-3)
    return g, ge, o, (src, rec)


def ws_bytes(lib, g, ge, o, op):
    n = ctypes.c_size_t(0)
    st = lib.fwi_workspace_bytes(ctypes.byref(g), ctypes.byref(ge) if ge is not None else None,
                                 ctypes.byref(o) if o is not None else None, op, ctypes.byref(n))
    return st, n.value


def test_workspace_sizes(lib):
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, keep = _structs()
    sizes = {}
    for op in range(6):
        st, n = ws_bytes(lib, g, ge, o, op)
        assert st == L.FWI_OK, lib.fwi_last_error()
        sizes[op] = n
    # the gradient holds the per-step sponge checkpoints: >= ns * nt * sponge cells * 4 B
    P, nz, nx, nt, ns = 10, 30, 40, 100, 2
    nband = 2 * P * (nx + 2 * P) + 2 * P * nz
    assert sizes[L.FWI_OP_GRADIENT] >= ns * nt * nband * 4
    assert sizes[L.FWI_OP_FORWARD] < sizes[L.FWI_OP_FORWARD_SAVE] <= sizes[L.FWI_OP_GRADIENT]
    # more shots, more workspace
    g2, ge2, o2, keep2 = _structs(ns=2, nt=200)
    assert ws_bytes(lib, g2, ge2, o2, L.FWI_OP_GRADIENT)[1] > sizes[L.FWI_OP_GRADIENT]


@pytest.mark.parametrize("field,value,code", [
    ("ndim", 4, 1), ("ny", 2, 1), ("nz", 0, 1), ("nt", 1, 1), ("sponge", 0, 1), ("dx", 0.0, 1),
    ("dt", -1.0, 1), ("refl", 1.0, 1), ("vref", 0.0, 1)])
def test_bad_grid_rejected(lib, field, value, code):
    g, ge, o, keep = _structs()
    setattr(g, field, value)
    st, _ = ws_bytes(lib, g, ge, o, 2)
    assert st == code
    assert len(lib.fwi_last_error()) > 0


@pytest.mark.parametrize("field,value", [("misfit", 7), ("illum_mode", 3), ("hmax", 13),
                                         ("hmax", -2), ("precond", 5), ("eps", 0.0), ("ckpt", 2),
                                         ("snap_prec", 3), ("snap_interval", -1), ("hess_v6", 2)])
def test_bad_options_rejected(lib, field, value):
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, keep = _structs()
    setattr(o, field, value)
    st, _ = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
    assert st == L.FWI_ERR_INVALID_ARG


def test_snapshot_workspace_sizes(lib):
    """Snapshot checkpoints replace the per-level sponge band by about sqrt(nt)
    whole fields: 2 fields per snapshot (F32) or 1 (16-bit), plus K - 1 segment
    slots. Long runs need far less workspace than the sponge mode."""
    from paper_1406_1864_gb300 import _lib as L
    nt, ns = 4000, 2
    g, ge, o, keep = _structs(nz=60, nx=80, nt=nt, ns=ns)
    sponge = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)[1]
    o.ckpt = L.FWI_CKPT_SNAPSHOT
    sizes = {}
    for prec in (L.FWI_SNAP_F32, L.FWI_SNAP_BF16, L.FWI_SNAP_F16S):
        o.snap_prec = prec
        st, n = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
        assert st == L.FWI_OK, lib.fwi_last_error()
        sizes[prec] = n
    assert sizes[L.FWI_SNAP_F32] < sponge / 4
    assert sizes[L.FWI_SNAP_BF16] == sizes[L.FWI_SNAP_F16S] < sizes[L.FWI_SNAP_F32]
    # K = ceil(sqrt(4000)) = 64 -> 63 snapshots of 2 fields; the F32 and 16-bit
    # plans differ by the snapshots' bytes (less the 16-bit maxima)
    nck = (nt - 1 + 63) // 64
    diff = sizes[L.FWI_SNAP_F32] - sizes[L.FWI_SNAP_BF16]
    field_all_shots = diff / (nck * 2 * 2)
    assert field_all_shots > ns * 60 * 80 and field_all_shots < ns * 4 * (60 + 40) * (80 + 100)
    # a longer interval keeps fewer snapshots but more segment slots
    o.snap_prec = L.FWI_SNAP_F32
    o.snap_interval = 8
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)[1] > sizes[L.FWI_SNAP_F32]
    # forward without save and the other forward-only calls keep nothing
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_FORWARD)[1] < sizes[L.FWI_SNAP_BF16]


def test_offset_precond_needs_hmax(lib):
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, keep = _structs()
    o.hmax, o.precond = -1, L.FWI_PRECOND_OFFSET
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)[0] == L.FWI_ERR_INVALID_ARG
    o.precond = L.FWI_PRECOND_ILLUM
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_OFFSET_HESSIAN)[0] == L.FWI_ERR_INVALID_ARG


def test_call_argument_errors_before_any_device_work(lib):
    """Entry points reject bad coordinates / NULL pointers / small workspaces
    before they queue anything (these return without touching a GPU)."""
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, (src, rec) = _structs()
    src[0, 0] = 30  # row out of range
    st = lib.fwi_forward(ctypes.byref(g), ctypes.byref(ge), None, ctypes.c_void_p(1),
                         ctypes.c_void_p(1), 0, ctypes.c_void_p(256), 1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG and b"outside" in lib.fwi_last_error()
    src[0, 0] = 0
    st = lib.fwi_forward(ctypes.byref(g), ctypes.byref(ge), None, None, ctypes.c_void_p(1), 0,
                         ctypes.c_void_p(256), 1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG
    st = lib.fwi_forward(ctypes.byref(g), ctypes.byref(ge), None, ctypes.c_void_p(1),
                         ctypes.c_void_p(1), 0, ctypes.c_void_p(256), 16, None)
    assert st == L.FWI_ERR_NOMEM
    st = lib.fwi_forward(ctypes.byref(g), ctypes.byref(ge), None, ctypes.c_void_p(1),
                         ctypes.c_void_p(1), 0, ctypes.c_void_p(8), 1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG  # misaligned workspace
    ge.src = None
    st = lib.fwi_forward(ctypes.byref(g), ctypes.byref(ge), None, ctypes.c_void_p(1),
                         ctypes.c_void_p(1), 0, ctypes.c_void_p(256), 1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG


def test_born_workspace_and_errors(lib):
    """Born modelling keeps u and du (four wavefield buffers); the
    Gauss-Newton product adds the Born traces and the backward pass's
    state, the same as a gradient without the illumination. Both take only
    sponge checkpoints and reject NULL inputs before any device work."""
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, keep = _structs()
    st, fwd = ws_bytes(lib, g, ge, None, L.FWI_OP_FORWARD)
    st1, born = ws_bytes(lib, g, ge, None, L.FWI_OP_BORN)
    st2, hvp = ws_bytes(lib, g, ge, None, L.FWI_OP_GN_HVP)
    st3, grad = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
    assert st == st1 == st2 == st3 == L.FWI_OK, lib.fwi_last_error()
    nzp, nxp = 30 + 20, 40 + 20
    assert born >= fwd + 2 * 2 * nzp * nxp * 4   # du^n, du^{n-1} for 2 shots
    assert born < hvp and hvp >= grad - 30 * 40 * 4 * 2
    o.ckpt = L.FWI_CKPT_SNAPSHOT
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_GN_HVP)[0] == L.FWI_ERR_INVALID_ARG
    assert ws_bytes(lib, g, ge, None, L.FWI_OP_PM_HESSIAN + 1)[0] == L.FWI_ERR_INVALID_ARG
    st = lib.fwi_born(ctypes.byref(g), ctypes.byref(ge), None, ctypes.c_void_p(1), None, ctypes.c_void_p(1),
                      ctypes.c_void_p(256), 1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG
    st = lib.fwi_gauss_newton_hvp(ctypes.byref(g), ctypes.byref(ge), None, ctypes.c_void_p(1), ctypes.c_void_p(1),
                                  None, ctypes.c_void_p(256), 1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG
    st = lib.fwi_born(ctypes.byref(g), ctypes.byref(ge), None, ctypes.c_void_p(1), ctypes.c_void_p(1),
                      ctypes.c_void_p(1), ctypes.c_void_p(256), 16, None)
    assert st == L.FWI_ERR_NOMEM


def test_misfit_workspace_and_header_constants(lib):
    """fwi_misfit keeps the forward fields and the residual traces (no
    checkpoints); the Python constants mirror the header's."""
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, keep = _structs()
    _, fwd = ws_bytes(lib, g, ge, None, L.FWI_OP_FORWARD)
    st, mis = ws_bytes(lib, g, ge, None, L.FWI_OP_MISFIT)
    _, grad = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
    assert st == L.FWI_OK
    assert mis >= fwd + 2 * 100 * 5 * 4 and mis < grad
    st = lib.fwi_misfit(ctypes.byref(g), ctypes.byref(ge), None, ctypes.c_void_p(1), ctypes.c_void_p(1), None,
                        ctypes.c_void_p(256), 1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG
    text = open(os.path.join(ROOT, "include", "fwi.h")).read()
    for name in ("FWI_CFL_LIMIT_2D", "FWI_CFL_LIMIT_3D"):
        m = re.search(r"#define\s+%s\s+([0-9.]+)f" % name, text)
        assert m and float(m.group(1)) == getattr(L, name), name
    m = re.search(r"FWI_OP_MISFIT\s*=\s*(\d+)", text)
    assert int(m.group(1)) == L.FWI_OP_MISFIT


def test_receiver_factor_workspace_and_errors(lib):
    """The Green's-function factor models the nrec receivers as sources
    without receivers (an offset-Hessian pass) plus their wavelets; the
    receiver preconditioning holds the product of scale and factor. Moving
    spreads and NULL outputs are refused before any device work."""
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, (src, rec) = _structs(ns=2, nrec=5)
    o.hmax = 2
    st, rf = ws_bytes(lib, g, ge, o, L.FWI_OP_RECEIVER_FACTOR)
    assert st == L.FWI_OK, lib.fwi_last_error()
    nzp, nxp = 30 + 20, 40 + 20
    assert rf >= 2 * 5 * nzp * nxp * 4 + 5 * 100 * 4   # u^n, u^{n-1} of 5 sources, their wavelets
    st, pr = ws_bytes(lib, g, None, None, L.FWI_OP_PRECONDITION_RECEIVER)
    assert st == L.FWI_OK and pr >= 13 * 30 * 40 * 4
    out = ctypes.c_void_p(256)
    st = lib.fwi_receiver_factor(ctypes.byref(g), ctypes.byref(ge), None, L.FWI_RECV_PLESSIX_MULDER, None, None,
                                 None, 0, None)
    assert st == L.FWI_ERR_INVALID_ARG
    rec[1, 0, 2] += 1  # shot 1 records elsewhere
    for kind in (L.FWI_RECV_PLESSIX_MULDER, L.FWI_RECV_GREEN):
        st = lib.fwi_receiver_factor(ctypes.byref(g), ctypes.byref(ge), None, kind, ctypes.c_void_p(1), out,
                                     ctypes.c_void_p(256), 1 << 40, None)
        assert st == L.FWI_ERR_INVALID_ARG and b"fixed spread" in lib.fwi_last_error()
    rec[1, 0, 2] -= 1
    st = lib.fwi_receiver_factor(ctypes.byref(g), ctypes.byref(ge), None, 7, None, out, None, 0, None)
    assert st == L.FWI_ERR_INVALID_ARG
    st = lib.fwi_precondition_receiver(ctypes.byref(g), ctypes.c_void_p(1), ctypes.c_void_p(1), L.FWI_PRECOND_OFFSET,
                                       4, ctypes.c_void_p(1), 3, ctypes.c_float(1e-3), ctypes.c_void_p(1),
                                       ctypes.c_void_p(256), 1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG  # 3 factor planes for 5 offsets


def test_extended_operator_workspace_and_errors(lib):
    """The extended Born pass holds u, du and the 13 planes of its scattering
    strengths; extended migration the gradient's state plus 13 image planes.
    Both refuse hext outside 0..6, snapshot checkpoints and NULL inputs."""
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, keep = _structs()
    _, born = ws_bytes(lib, g, ge, None, L.FWI_OP_BORN)
    st, eb = ws_bytes(lib, g, ge, None, L.FWI_OP_EXT_BORN)
    assert st == L.FWI_OK and eb >= born + 13 * 50 * 60 * 4
    _, fs = ws_bytes(lib, g, ge, None, L.FWI_OP_FORWARD_SAVE)
    st, em = ws_bytes(lib, g, ge, None, L.FWI_OP_EXT_MIGRATION)
    assert st == L.FWI_OK and em >= fs + 13 * 50 * 60 * 4
    o.ckpt = L.FWI_CKPT_SNAPSHOT
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_EXT_MIGRATION)[0] == L.FWI_ERR_INVALID_ARG
    p1 = ctypes.c_void_p(1)
    for hext in (-1, 7):
        st = lib.fwi_extended_born(ctypes.byref(g), ctypes.byref(ge), None, hext, p1, p1, p1, ctypes.c_void_p(256),
                                   1 << 40, None)
        assert st == L.FWI_ERR_INVALID_ARG
        st = lib.fwi_extended_migration(ctypes.byref(g), ctypes.byref(ge), None, hext, p1, p1, p1,
                                        ctypes.c_void_p(256), 1 << 40, None)
        assert st == L.FWI_ERR_INVALID_ARG
    st = lib.fwi_extended_migration(ctypes.byref(g), ctypes.byref(ge), None, 2, p1, p1, None, ctypes.c_void_p(256),
                                    1 << 40, None)
    assert st == L.FWI_ERR_INVALID_ARG


def test_selftest_wait_argument_errors(lib):
    """The bounded-wait self-test checks its arguments before any device work."""
    from paper_1406_1864_gb300 import _lib as L
    assert lib.fwi_selftest_wait(0, ctypes.c_void_p(256), 256, None) == L.FWI_ERR_INVALID_ARG
    assert lib.fwi_selftest_wait(20000000, ctypes.c_void_p(256), 256, None) == L.FWI_ERR_INVALID_ARG
    assert lib.fwi_selftest_wait(1000, None, 256, None) == L.FWI_ERR_INVALID_ARG
    assert lib.fwi_selftest_wait(1000, ctypes.c_void_p(8), 256, None) == L.FWI_ERR_INVALID_ARG
    assert lib.fwi_selftest_wait(1000, ctypes.c_void_p(256), 16, None) == L.FWI_ERR_NOMEM


def test_product_path_does_not_import_the_oracle():
    import subprocess
    import sys
    code = ("import sys; import paper_1406_1864_gb300.fwi, paper_1406_1864_gb300.workloads; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    out = subprocess.check_output([sys.executable, "-c", code], cwd=ROOT).decode().strip()
    assert out == "False"
    for f in glob.glob(os.path.join(ROOT, "paper_1406_1864_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".h", ".cuh")):
            txt = open(f).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f


def test_batch_workspace_and_errors(lib):
    """A batch of models lays the models' gradient workspaces end to end; it
    refuses mismatched nt, snapshot checkpoints with several models, and a
    model count outside 1..FWI_BATCH_MAX (all before any device work)."""
    from paper_1406_1864_gb300 import _lib as L
    (g1, ge1, o, k1), (g2, ge2, _, k2) = _structs(nz=30, nx=40), _structs(nz=50, nx=70, ns=2)
    singles = [ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)[1] for g, ge in ((g1, ge1), (g2, ge2))]
    G = (L.FwiGrid * 2)(g1, g2)
    GE = (L.FwiGeometry * 2)(ge1, ge2)
    n = ctypes.c_size_t(0)
    assert lib.fwi_batch_workspace_bytes(2, G, GE, ctypes.byref(o), ctypes.byref(n)) == L.FWI_OK
    align = lambda x: (x + 255) // 256 * 256
    assert n.value == align(singles[0]) + align(singles[1])
    assert lib.fwi_batch_workspace_bytes(1, G, GE, ctypes.byref(o), ctypes.byref(n)) == L.FWI_OK
    assert n.value == align(singles[0])
    for bad in (0, L.FWI_BATCH_MAX + 1):
        assert lib.fwi_batch_workspace_bytes(bad, G, GE, ctypes.byref(o), ctypes.byref(n)) == L.FWI_ERR_INVALID_ARG
    G[1].nt = 99
    assert lib.fwi_batch_workspace_bytes(2, G, GE, ctypes.byref(o), ctypes.byref(n)) == L.FWI_ERR_INVALID_ARG
    assert b"nt" in lib.fwi_last_error()
    G[1].nt = G[0].nt
    o.ckpt = L.FWI_CKPT_SNAPSHOT
    assert lib.fwi_batch_workspace_bytes(2, G, GE, ctypes.byref(o), ctypes.byref(n)) == L.FWI_ERR_INVALID_ARG
    assert lib.fwi_batch_workspace_bytes(1, G, GE, ctypes.byref(o), ctypes.byref(n)) == L.FWI_OK
    o.ckpt = L.FWI_CKPT_SPONGE
    G[1].nz = 0
    assert lib.fwi_batch_workspace_bytes(2, G, GE, ctypes.byref(o), ctypes.byref(n)) == L.FWI_ERR_INVALID_ARG
    assert b"model 1" in lib.fwi_last_error()


def test_3d_workspace_and_options(lib):
    """3-D plans: snapshot checkpoints required for gradients and for forward
    modelling that keeps checkpoints (all shots in one group); the offset
    Hessian (gradients, its diagonal) adds its hmax + 1 sums of the physical
    grid and needs hmax >= 0; shot groups bound the workspace (one group's
    fields and snapshots); forward modelling needs no checkpoints."""
    from paper_1406_1864_gb300 import _lib as L
    g = L.FwiGrid(3, 20, 24, 28, 10.0, 1e-3, 100, 8, 3000.0, 0.05)
    ns, nrec = 4, 6
    src = np.zeros((ns, 3), np.int32)
    src[:, 1] = 12
    src[:, 2] = [3, 9, 15, 21]
    rec = np.zeros((ns, nrec, 3), np.int32)
    rec[:, :, 1] = 12
    rec[:, :, 2] = np.arange(nrec) * 4
    ge = L.FwiGeometry(ns, nrec, src.ctypes.data, rec.ctypes.data, 1)
    o = L.FwiOptions(0, 0, -1, 1, 1e-3)
    st, _ = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
    assert st == L.FWI_ERR_INVALID_ARG and b"SNAPSHOT" in lib.fwi_last_error()
    o.ckpt = L.FWI_CKPT_SNAPSHOT
    st, full = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
    assert st == L.FWI_OK, lib.fwi_last_error()
    o.shot_group = 1
    st, one = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
    assert st == L.FWI_OK and one < full / 2
    o.snap_prec = L.FWI_SNAP_BF16
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)[1] < one
    st, fw = ws_bytes(lib, g, ge, o, L.FWI_OP_FORWARD)
    assert st == L.FWI_OK and fw < one
    st, plain = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
    nphys = 20 * 24 * 28
    o.hmax = 2
    st, with_h = ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)
    assert st == L.FWI_OK, lib.fwi_last_error()
    assert with_h - plain == -(-3 * nphys * 4 // 256) * 256
    o.hmax = 13
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)[0] == L.FWI_ERR_INVALID_ARG
    o.hmax, o.precond = -1, L.FWI_PRECOND_OFFSET
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)[0] == L.FWI_ERR_INVALID_ARG
    o.precond = L.FWI_PRECOND_ILLUM
    # forward with checkpoints keeps every shot's snapshots: one group only
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_FORWARD_SAVE)[0] == L.FWI_ERR_INVALID_ARG
    o.shot_group = 0
    st, fs = ws_bytes(lib, g, ge, o, L.FWI_OP_FORWARD_SAVE)
    assert st == L.FWI_OK and fs > one
    o.ckpt = L.FWI_CKPT_SPONGE
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_FORWARD_SAVE)[0] == L.FWI_ERR_INVALID_ARG
    o.ckpt = L.FWI_CKPT_SNAPSHOT
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_OFFSET_HESSIAN)[0] == L.FWI_ERR_INVALID_ARG
    assert b"hmax >= 0" in lib.fwi_last_error()
    o.hmax = 3
    st, oh = ws_bytes(lib, g, ge, o, L.FWI_OP_OFFSET_HESSIAN)
    assert st == L.FWI_OK, lib.fwi_last_error()
    assert oh < fs  # no snapshots
    o.hmax = -1
    # the elementwise division: status word and maximum only
    assert ws_bytes(lib, g, None, None, L.FWI_OP_PRECONDITION) == (L.FWI_OK, 256)
    one_f = ctypes.c_void_p(256)
    st = lib.fwi_precondition(ctypes.byref(g), None, one_f, L.FWI_PRECOND_OFFSET, 2, ctypes.c_float(1e-3), one_f,
                              None, 0, None)
    assert st == L.FWI_ERR_INVALID_ARG and b"NULL" in lib.fwi_last_error()
    st = lib.fwi_precondition(ctypes.byref(g), one_f, one_f, L.FWI_PRECOND_OFFSET, 13, ctypes.c_float(1e-3), one_f,
                              None, 0, None)
    assert st == L.FWI_ERR_INVALID_ARG and b"hmax" in lib.fwi_last_error()
    o.shot_group = -1
    assert ws_bytes(lib, g, ge, o, L.FWI_OP_GRADIENT)[0] == L.FWI_ERR_INVALID_ARG


def test_3d_autotune_set_checks_the_variants(lib):
    """fwi_autotune_set on a 3-D problem accepts the compiled variants (3
    forward, 4 backward) and z-segment counts >= 0 and refuses others, before
    any device work; fwi_autotune_reset forgets the choice."""
    from paper_1406_1864_gb300 import _lib as L
    g = L.FwiGrid(3, 20, 24, 28, 10.0, 1e-3, 100, 8, 3000.0, 0.05)
    src = np.array([[0, 12, 3]], np.int32)
    rec = np.array([[[0, 12, 8], [0, 12, 16]]], np.int32)
    ge = L.FwiGeometry(1, 2, src.ctypes.data, rec.ctypes.data, 1)
    o = L.FwiOptions(0, 0, -1, 1, 1e-3)
    o.ckpt = L.FWI_CKPT_SNAPSHOT
    for fv, bv, ok in ((0, 0, True), (2, 3, True), (3, 0, False), (0, 4, False), (-1, 0, False)):
        ch = (ctypes.c_int * 4)(fv, 1, bv, 1)
        st = lib.fwi_autotune_set(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(o), ch)
        assert (st == L.FWI_OK) == ok, (fv, bv, st)
    # the 3-D chunks are z-segments per column: 0 (chosen per launch shape) or more
    for fs, bs, ok in ((0, 0, True), (3, 40, True), (-1, 0, False), (0, -2, False)):
        ch = (ctypes.c_int * 4)(0, fs, 0, bs)
        st = lib.fwi_autotune_set(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(o), ch)
        assert (st == L.FWI_OK) == ok, (fs, bs, st)
    assert lib.fwi_autotune_reset() == L.FWI_OK


def test_3d_forward_save_and_adjoint_apply_errors(lib):
    """3-D fwi_forward(save = 1) and fwi_adjoint_apply reject, before any
    device work: sponge checkpoints, shot groups smaller than the shots,
    NULL outputs and small workspaces."""
    from paper_1406_1864_gb300 import _lib as L
    g = L.FwiGrid(3, 20, 24, 28, 10.0, 1e-3, 100, 8, 3000.0, 0.05)
    src = np.array([[0, 12, 3], [0, 12, 20]], np.int32)
    rec = np.array([[[0, 12, 8], [0, 12, 16]]] * 2, np.int32)
    ge = L.FwiGeometry(2, 2, src.ctypes.data, rec.ctypes.data, 1)
    o = L.FwiOptions(0, 0, -1, 1, 1e-3)
    p1, big = ctypes.c_void_p(256), 1 << 40

    def fwd(opts, seis=ctypes.c_void_p(256), nbytes=big):
        return lib.fwi_forward(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(opts) if opts else None,
                               ctypes.c_void_p(256), seis, 1, p1, nbytes, None)

    assert fwd(None) == L.FWI_ERR_INVALID_ARG and b"SNAPSHOT" in lib.fwi_last_error()
    assert fwd(o) == L.FWI_ERR_INVALID_ARG                      # sponge checkpoints
    o.ckpt = L.FWI_CKPT_SNAPSHOT
    o.shot_group = 1
    assert fwd(o) == L.FWI_ERR_INVALID_ARG and b"shot_group" in lib.fwi_last_error()
    o.shot_group = 0
    assert fwd(o, seis=None) == L.FWI_ERR_INVALID_ARG
    assert fwd(o, nbytes=16) == L.FWI_ERR_NOMEM
    st = lib.fwi_adjoint_apply(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(o), ctypes.c_void_p(256),
                               ctypes.c_void_p(256), None, p1, big, None)
    assert st == L.FWI_ERR_INVALID_ARG                          # grad is NULL
    st = lib.fwi_adjoint_apply(ctypes.byref(g), ctypes.byref(ge), ctypes.byref(o), ctypes.c_void_p(256),
                               ctypes.c_void_p(256), ctypes.c_void_p(256), p1, 16, None)
    assert st == L.FWI_ERR_NOMEM


def test_forward_noalloc_argument_errors(lib):
    """fwi_forward_noalloc rejects bad arguments before any device work and
    before it looks up its scratch array's address: on this GPU-less host a
    call that got that far would fail with a CUDA error instead."""
    from paper_1406_1864_gb300 import _lib as L
    g, ge, o, (src, rec) = _structs()
    p1 = ctypes.c_void_p(256)

    def call(grid=g, geom=ge, v=p1, seis=p1):
        return lib.fwi_forward_noalloc(ctypes.byref(grid) if grid is not None else None,
                                       ctypes.byref(geom) if geom is not None else None, v, seis, None)

    assert call(grid=None) == L.FWI_ERR_INVALID_ARG and b"grid is NULL" in lib.fwi_last_error()
    g3 = L.FwiGrid(3, 20, 24, 28, 10.0, 1e-3, 100, 8, 3000.0, 0.05)
    assert call(grid=g3) == L.FWI_ERR_INVALID_ARG and b"2-D" in lib.fwi_last_error()
    assert call(geom=None) == L.FWI_ERR_INVALID_ARG and b"geometry is NULL" in lib.fwi_last_error()
    assert call(v=None) == L.FWI_ERR_INVALID_ARG and b"NULL" in lib.fwi_last_error()
    assert call(seis=None) == L.FWI_ERR_INVALID_ARG and b"NULL" in lib.fwi_last_error()
    src[0, 0] = 30  # row out of range
    assert call() == L.FWI_ERR_INVALID_ARG and b"outside" in lib.fwi_last_error()
    src[0, 0] = 0
    big = L.FwiGrid(2, 1500, 1, 1500, 10.0, 1e-3, 10, 20, 3000.0, 0.05)
    assert call(grid=big) == L.FWI_ERR_NOMEM and b"scratch" in lib.fwi_last_error()
