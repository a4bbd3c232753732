"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports every
function that include/dg.h declares, and rejects invalid arguments before touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_10885_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dg_setup", "dg_apply_residual", "dg_apply_jacobian", "dg_destroy", "dg_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1711_10885_gb300 import dg
    assert set(dg.EXPORTED) <= set(declared_functions())


def test_penalty_conventions(lib):
    lib.dg_penalty_sigma.restype = ctypes.c_double
    lib.dg_penalty_sigma.argtypes = [ctypes.c_int32, ctypes.c_int32]
    assert lib.dg_penalty_sigma(3, 0) == 24.0  # 2k(k+1): 24/h for k = 3 and D = 1
    assert lib.dg_penalty_sigma(7, 1) == 2.0 * 7 * 9  # alpha p (p + d - 1), alpha = 2


def test_setup_rejects_invalid_arguments_on_host():
    from paper_1711_10885_gb300 import dg
    mesh = dg.dg_mesh()
    for r in range(3):
        mesh.lo[r], mesh.hi[r], mesh.n[r] = 0.0, 1.0, 2
    co = dg.dg_coeffs()
    co.D_const, co.c, co.sigma = 1.0, 1.0, 4.0
    h = ctypes.c_void_p()

    def setup(k, mesh=mesh, co=co):
        return dg.lib.dg_setup(ctypes.byref(mesh), k, ctypes.byref(co), None, None, None, ctypes.byref(h))

    assert setup(0) == -1 and b"degree" in dg.lib.dg_last_error()
    assert setup(11) == -1
    bad = dg.dg_coeffs()
    bad.D_const, bad.c, bad.sigma = -1.0, 1.0, 4.0
    assert setup(2, co=bad) == -1 and b"D_T" in dg.lib.dg_last_error()
    bad.D_const = float("nan")
    assert setup(2, co=bad) == -1
    bad.D_const, bad.sigma = 1.0, float("inf")
    assert setup(2, co=bad) == -1
    m2 = dg.dg_mesh()
    for r in range(3):
        m2.lo[r], m2.hi[r], m2.n[r] = 0.0, 1.0, 2
    m2.n[1] = 0
    assert setup(2, mesh=m2) == -1
    m2.n[1], m2.hi[2] = 2, 0.0
    assert setup(2, mesh=m2) == -1
    assert dg.lib.dg_setup(ctypes.byref(mesh), 2, ctypes.byref(co), None, None, None, None) == -1
    assert h.value is None


def test_setup_ex_rejects_invalid_transport_options_on_host():
    from paper_1711_10885_gb300 import dg
    mesh = dg.dg_mesh()
    for r in range(3):
        mesh.lo[r], mesh.hi[r], mesh.n[r] = 0.0, 1.0, 2
    co = dg.dg_coeffs()
    co.D_const, co.c, co.sigma = 1.0, 0.0, 4.0
    h = ctypes.c_void_p()

    def setup(k, ext):
        return dg.lib.dg_setup_ex(ctypes.byref(mesh), k, ctypes.byref(co), None, None, ctypes.byref(ext), None,
                                  ctypes.byref(h))

    ext = dg.dg_setup_ext()
    ext.m = 5  # k+2: only k+1 and k+3 are offered
    assert setup(3, ext) == -1 and b"m must be" in dg.lib.dg_last_error()
    ext.m, ext.velocity = 0, 7
    assert setup(3, ext) == -1 and b"velocity" in dg.lib.dg_last_error()
    ext.velocity = dg.DG_VELOCITY_POINTS  # needs both point arrays
    assert setup(3, ext) == -1 and b"b_qp" in dg.lib.dg_last_error()
    ext.velocity = dg.DG_VELOCITY_TAYLOR_GREEN
    assert setup(9, ext) == -1 and b"k <= 8" in dg.lib.dg_last_error()
    ext.velocity, ext.periodic[1] = dg.DG_VELOCITY_CONSTANT, 2
    assert setup(3, ext) == -1 and b"periodic" in dg.lib.dg_last_error()
    assert h.value is None


def test_time_stepping_entry_points_reject_null_arguments_on_host():
    from paper_1711_10885_gb300 import dg
    assert dg.lib.dg_project(None, None, None, None) == -1
    assert dg.lib.dg_rk_stage(None, None, None, None, 0.0, 1.0, 0.1, 0, None) == -1
    assert dg.lib.dg_ssprk2(None, None, 0.1, 1, 0, None) == -1


def test_setup_ex_rejects_bad_tensors_and_jacobians_on_host():
    from paper_1711_10885_gb300 import dg
    mesh = dg.dg_mesh()
    for r in range(3):
        mesh.lo[r], mesh.hi[r], mesh.n[r] = 0.0, 1.0, 1
    co = dg.dg_coeffs()
    co.D_const, co.c, co.sigma = 1.0, 0.0, 4.0
    h = ctypes.c_void_p()
    ext = dg.dg_setup_ext()
    bad = (ctypes.c_double * 6)(1.0, 1.0, 1.0, 2.0, 0.0, 0.0)  # indefinite: xy entry too large
    ext.D_tensor = ctypes.cast(bad, dg._dp)
    rc = dg.lib.dg_setup_ex(ctypes.byref(mesh), 2, ctypes.byref(co), None, None, ctypes.byref(ext), None,
                            ctypes.byref(h))
    assert rc == -1 and b"positive definite" in dg.lib.dg_last_error()
    ext.D_tensor = dg._dp()
    ext.velocity = dg.DG_VELOCITY_TAYLOR_GREEN
    J = (ctypes.c_double * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    ext.jacobian = ctypes.cast(J, dg._dp)
    rc = dg.lib.dg_setup_ex(ctypes.byref(mesh), 2, ctypes.byref(co), None, None, ctypes.byref(ext), None,
                            ctypes.byref(h))
    assert rc == -1 and b"constant velocity" in dg.lib.dg_last_error()
    assert h.value is None


def test_setup_ex_rejects_bad_boundary_types_on_host():
    from paper_1711_10885_gb300 import dg
    mesh = dg.dg_mesh()
    for r in range(3):
        mesh.lo[r], mesh.hi[r], mesh.n[r] = 0.0, 1.0, 2
    co = dg.dg_coeffs()
    co.D_const, co.c, co.sigma = 1.0, 0.0, 4.0
    h = ctypes.c_void_p()
    ext = dg.dg_setup_ext()
    ext.bc_type[3] = 5
    rc = dg.lib.dg_setup_ex(ctypes.byref(mesh), 2, ctypes.byref(co), None, None, ctypes.byref(ext), None,
                            ctypes.byref(h))
    assert rc == -1 and b"bc_type" in dg.lib.dg_last_error()
    ext.bc_type[3] = dg.DG_BC_OUTFLOW
    D = (ctypes.c_double * 6)(1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    ext.D_qp = ctypes.cast(D, dg._dp)  # D_face missing
    rc = dg.lib.dg_setup_ex(ctypes.byref(mesh), 2, ctypes.byref(co), None, None, ctypes.byref(ext), None,
                            ctypes.byref(h))
    assert rc == -1 and b"D_face" in dg.lib.dg_last_error()
    assert h.value is None


def test_operator_marshals_every_option():
    """The binding turns every option into the C structs (on a machine without a GPU the call then fails in
    CUDA, which the binding reports as DGError; a marshalling mistake would raise something else)."""
    import numpy as np
    from paper_1711_10885_gb300 import dg
    n, k, m = (2, 1, 1), 1, 4
    nc = 2
    eye6 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    kw = dict(b=(0.5, 0.0, 0.0), c=0.3, m=m, periodic=(0, 1, 0), velocity="points",
              b_qp=np.zeros((nc, m ** 3, 3)), b_face=np.zeros((nc, 6, m ** 2)), jacobian=np.eye(3) * 0.5,
              D_qp=np.tile(eye6, (nc, m ** 3, 1)), D_face=np.tile(eye6, (nc, 6, m ** 2, 1)),
              c_qp=np.ones((nc, m ** 3)), bc=("dirichlet", "outflow", "neumann", "neumann", 0, 2),
              f_qp=np.ones(nc * m ** 3), g_qp=[np.zeros(m * m)] * 6, stream=0)
    try:
        op = dg.Operator(n, k, 1.0, **kw)
    except dg.DGError:
        return
    op.close()  # a GPU was present: the handle was built


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets of include/dg.h (compiled here with gcc)."""
    import os
    import subprocess
    from paper_1711_10885_gb300 import dg
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = {"dg_mesh": dg.dg_mesh, "dg_coeffs": dg.dg_coeffs, "dg_bc": dg.dg_bc, "dg_setup_ext": dg.dg_setup_ext,
               "dg_solve_opts": dg.dg_solve_opts, "dg_solve_stats": dg.dg_solve_stats,
               "dg_mlp_train_opts": dg.dg_mlp_train_opts, "dg_mlp_train_stats": dg.dg_mlp_train_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def header_constants():
    """Integer constants of include/dg.h: enumerators with explicit values and plain integer #defines."""
    text = open(os.path.join(ROOT, "include", "dg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body in re.findall(r"\benum\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"\b(DG_\w+)\s*=\s*(-?\d+)", body):
            out[name] = int(val)
    for name, val in re.findall(r"^\s*#define\s+(DG_\w+)\s+(-?\d+)\s*$", text, flags=re.M):
        out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    from paper_1711_10885_gb300 import dg
    consts = header_constants()
    # every option family of the header is visible in the binding, with the header's values
    for prefix in ("DG_F", "DG_SOLVE_", "DG_PRECOND_", "DG_BJ_", "DG_BC_", "DG_VELOCITY_"):
        names = [n for n in consts if n.startswith(prefix) and not n.startswith("DG_ERR_")]
        assert names, prefix
        for n in names:
            assert getattr(dg, n) == consts[n], n
    for n, v in consts.items():
        if hasattr(dg, n):
            assert getattr(dg, n) == v, n


def declared_prototypes():
    """(name, return type, [parameter types]) of every function include/dg.h declares."""
    text = open(os.path.join(ROOT, "include", "dg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"^\s*#.*$", "", text, flags=re.M)
    out = []
    for ret, name, params in re.findall(r"([A-Za-z_][\w\s\*]*?)\b(dg_\w+)\s*\(([^)]*)\)\s*;", text):
        ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        out.append((name, " ".join(ret.split()), ps))
    return out


def null_args(params):
    vals = []
    for p in params:
        if "*" in p:
            vals.append(ctypes.c_void_p(None))
        elif "uint64_t" in p:
            vals.append(ctypes.c_uint64(0))
        elif "int64_t" in p:
            vals.append(ctypes.c_int64(0))
        elif "int32_t" in p:
            vals.append(ctypes.c_int32(0))
        elif "double" in p:
            vals.append(ctypes.c_double(0.0))
        elif "float" in p:
            vals.append(ctypes.c_float(0.0))
        else:
            raise AssertionError(f"unmapped parameter type: {p}")
    return vals


def test_every_entry_point_rejects_null_handles_without_touching_the_device(lib):
    """Every call with null handles, null pointers and zero sizes returns an error code and a message, except the
    destroy calls, for which null is a no-op; nothing crashes and no device work starts."""
    lib.dg_last_error.restype = ctypes.c_char_p
    protos = declared_prototypes()
    assert len(protos) >= 30
    for name, ret, params in protos:
        if name in ("dg_last_error", "dg_penalty_sigma"):
            continue
        assert ret.endswith("int"), (name, ret)
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        rc = fn(*null_args(params))
        if name.endswith("_destroy"):
            assert rc == 0, name
        else:
            assert rc < 0, name
            assert lib.dg_last_error(), name
