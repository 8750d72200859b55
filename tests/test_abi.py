"""The C-ABI library loads on a machine without a GPU and exports every
function that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("radon_fwd", "radon_adj", "mbir_grad", "mbir_solve", "tc_plan_create",
               "tc_plan_destroy", "tc_status_string"):
        assert fn in names


def test_library_exports_every_declared_symbol():
    from paper_2304_12934_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_2304_12934_gb300 import api
    L = api.load()
    assert L.tc_status_string(0) == b"ok"
    assert L.tc_status_string(-1) == b"invalid argument"
    assert L.tc_status_string(12345) == b"unknown status"


def test_invalid_geometry_rejected_on_host():
    """Argument checks run before any CUDA call."""
    from paper_2304_12934_gb300 import api
    L = api.load()
    h = ctypes.c_void_p()
    for n, a, d, os_, w in ((100, 10, 20, 2, 7), (64, 10, 21, 2, 7), (64, 0, 20, 2, 7),
                            (64, 10, 20, 3, 7), (64, 10, 20, 2, 9), (8, 10, 20, 2, 7)):
        g = api._Geom(n, a, d, ctypes.POINTER(ctypes.c_double)(), os_, w)
        assert L.tc_plan_create(ctypes.byref(g), 1, ctypes.byref(h)) == -1
        assert not h.value
    for delta in (float("nan"), float("inf"), 10.5, -11.0):  # |delta| <= D/2 = 10
        g = api._Geom(64, 10, 20, ctypes.POINTER(ctypes.c_double)(), 2, 7, delta)
        assert L.tc_plan_create(ctypes.byref(g), 1, ctypes.byref(h)) == -1
        assert not h.value
    assert L.radon_fwd(None, None, None, 1, None) == -1
    assert L.tc_plan_destroy(None) == 0


def test_product_path_does_not_import_oracle():
    for f in glob.glob(os.path.join(ROOT, "paper_2304_12934_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            src = open(f).read()
            assert "import oracle" not in src and "from oracle" not in src, f
            assert "radon_oracle" not in src, f


def test_restart_modes_map_to_the_abi_codes():
    from paper_2304_12934_gb300 import api
    assert api._restart_code(True) == 1 and api._restart_code(False) == 0
    assert api._restart_code("monotone") == 2
    with pytest.raises(ValueError):
        api._restart_code("sometimes")


def test_checkpoint_reader_rejects_bad_files_before_any_device_work(tmp_path):
    """A missing file, a foreign format and a truncated header are refused on
    the host (TC_ERR_INVALID_ARG) before the plan or a device buffer is used."""
    from paper_2304_12934_gb300 import api
    L = api.load()
    fake_plan = ctypes.create_string_buffer(1 << 16)   # never dereferenced on these paths
    st = api._SolveState()
    st.z = ctypes.addressof(ctypes.create_string_buffer(64))
    x = ctypes.create_string_buffer(64)
    bad = tmp_path / "bad.ckpt"
    for content in (None, b'{"format": "something-else", "version": 1}\n', b'{"format": "tc-mbir-ch'):
        if content is not None:
            bad.write_bytes(content)
        path = str(bad if content is not None else tmp_path / "missing.ckpt").encode()
        rc = L.tc_checkpoint_load(path, ctypes.addressof(fake_plan), ctypes.addressof(x), 1,
                                  ctypes.byref(st), None)
        assert rc == -1
    assert L.tc_checkpoint_save(None, None, None, 1, None, None) == -1


def test_solver_options_layout_matches_the_header():
    """The binding's mirror of tc_solve_opts / tc_solve_state has the fields
    the header declares, in order (a mismatch would shift every field)."""
    from paper_2304_12934_gb300 import api
    src = open(os.path.join(ROOT, "include", "nufft_radon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for cname, py in (("tc_solve_opts", api._SolveOpts), ("tc_solve_state", api._SolveState),
                      ("tc_geom", api._Geom), ("tc_prior", api._Prior)):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + cname + ";", src).group(1)
        names = re.findall(r"(\w+)\s*(?:\[\d+\])?\s*;", body)
        py_names = [f[0] for f in py._fields_]
        assert [n if n != "lambda" else "lam" for n in names] == py_names, (cname, names, py_names)


def test_solver_state_follows_an_exchange_of_z_and_g():
    """The solve may hand back state.z and state.g exchanged (a prior's solver
    form makes z_{k+1} where the gradient was); the binding's SolveState then
    swaps its two tensors to match, and refuses a pointer to neither."""
    torch = pytest.importorskip("torch")
    from paper_2304_12934_gb300 import api
    st = api.SolveState(torch.zeros(2, 4, 4))
    z0, g0 = st.z, st.g
    cs = st._c()
    cs.z, cs.g = g0.data_ptr(), z0.data_ptr()
    cs.t, cs.k = 3.5, 7
    st._load(cs)
    assert st.z is g0 and st.g is z0 and st.k == 7 and st.t == 3.5
    cs = st._c()
    st._load(cs)  # not exchanged: unchanged
    assert st.z is g0 and st.g is z0
    cs.z = torch.zeros(1).data_ptr()
    with pytest.raises(RuntimeError):
        st._load(cs)


def test_sfu_probe_rejects_bad_arguments_without_gpu():
    """tc_sfu_throughput checks its operation code and output pointer before
    touching the device."""
    from paper_2304_12934_gb300 import api
    L = api.load()
    out = ctypes.c_double()
    for op in (-1, 3, 99):
        assert L.tc_sfu_throughput(op, ctypes.byref(out), None) == -1
    assert L.tc_sfu_throughput(0, None, None) == -1
