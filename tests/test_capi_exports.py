"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/pocketvina.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pocketvina.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:pv_status|void|const char\s*\*)\s*\**\s*(pv_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pv_context_create", "pv_build_grids", "pv_ligand_create", "pv_dock", "pv_score",
                     "pv_score_backward", "pv_dock_result_destroy", "pv_grid_set_view", "pv_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2506_20043_gb300 as pv
    from paper_2506_20043_gb300 import _capi
    lib_path = pv.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) == set(_capi.SIGNATURES), set(_declared()) ^ set(_capi.SIGNATURES)


def test_binding_refuses_to_run_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_20043_gb300 import api
    with pytest.raises(api.PVError):
        api.Context(0)


def test_pocket_parameter_defaults_agree():
    # host-only entry point: the binding's defaults are the library's
    import dataclasses
    from paper_2506_20043_gb300 import _capi, api
    lib = _capi.load()
    p = _capi.pv_pocket_params()
    assert lib.pv_pocket_params_default(ctypes.byref(p)) == _capi.PV_OK
    q = api.PocketParams()
    for f in dataclasses.fields(q):
        assert getattr(p, f.name) == pytest.approx(getattr(q, f.name)), f.name
    assert lib.pv_pocket_params_default(None) == _capi.PV_ERR_ARG


def test_dock_params_layout_and_defaults_agree(tmp_path):
    """The binding's pv_dock_params has the C struct's size and field offsets (compiled with the
    host compiler from the header), and its defaults are the library's (host-only call)."""
    import dataclasses
    import shutil
    import subprocess
    from paper_2506_20043_gb300 import _capi, api
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    fields = [f[0] for f in _capi.pv_dock_params._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pocketvina.h"\nint main(void) {\n'
                    '  printf("%zu\\n", sizeof(pv_dock_params));\n' +
                    "".join(f'  printf("%zu\\n", offsetof(pv_dock_params, {f}));\n' for f in fields) +
                    "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(_capi.pv_dock_params)
    assert got[1:] == [getattr(_capi.pv_dock_params, f).offset for f in fields]
    lib = _capi.load()
    p = _capi.pv_dock_params()
    lib.pv_dock_params_default(ctypes.byref(p))
    q = api.DockParams()
    for f in dataclasses.fields(q):
        if f.name == "pair_keys":
            assert not p.pair_keys and q.pair_keys is None
            continue
        if f.name == "resume_state":
            assert not p.resume_state and p.resume_bytes == 0 and q.resume_state is None
            continue
        v = getattr(q, f.name)
        if f.name == "mode":
            v = _capi.PV_MODE_BATCHED
        assert getattr(p, f.name) == pytest.approx(float(v)), f.name
