"""CPU checks of the C ABI: the library loads, exports every entry point the
headers in include/ declare, and rejects invalid configurations on the host
before touching a GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(lbm\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_0908_3749_gb300 import lbm
    lib = lbm.load()
    names = _declared()
    assert {"lbm_create", "lbm_set_init", "lbm_step", "lbm_moments", "lbm_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


@pytest.mark.parametrize("change,code", [
    ({"nx": 0}, -1), ({"ny": 0}, -1), ({"dt": 0.0}, -1), ({"dx": -1.0}, -1),
    ({"dt": 1.0}, -1),                         # Courant number 6 dt/dx > 1
    ({"internal_dof": 3}, -2), ({"precision": 7}, -2),
    ({"s0": float("nan")}, -1), ({"bc0": ("periodic", None)}, -1),   # periodic on one side only
    ({"audit_every": -1}, -1),
    ({"bc0": ("eq", (1, 0, 0, 1), ("periodic", 0.0, 0.0))}, -1),      # split into periodic
    ({"bc0": ("extrap", None, ("eq", 0.0, 0.0))}, -1),               # far Dirichlet state missing
    ({"bc0": ("eq", (1, 0, 0, 1), ("reflect", float("inf"), 0.0))}, -1),
    ({"nx": 16384, "ny": 16448, "precision": "tc_tf32x3"}, -2),     # 2^32 elements: no TC form
])
def test_create_rejects_bad_configs_on_host(change, code):
    from paper_0908_3749_gb300 import lbm
    kw = dict(nx=8, ny=4, dx=0.01, dy=0.01, dt=1e-5, s=[1e5] * 16,
              bc=[("eq", (1, 0, 0, 1)), ("eq", (1, 0, 0, 1)), ("periodic", None), ("periodic", None)],
              precision="fp64", audit_every=0, internal_dof=0)
    for k, v in change.items():
        if k == "s0":
            kw["s"] = [v] + kw["s"][1:]
        elif k == "bc0":
            kw["bc"] = [v] + kw["bc"][1:]
        else:
            kw[k] = v
    cfg = lbm.make_config(**kw)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(cfg)
    assert ei.value.code == code
    assert lbm.lbm_last_error(None)


def test_launch_shape_entry_points_reject_null_context():
    from paper_0908_3749_gb300 import lbm
    lib = lbm.load()
    assert lib.lbm_set_step_blocks(None, 4) == lbm.LBM_ERR_INVALID
    assert lib.lbm_step_blocks(None) == -1
    assert lib.lbm_autotune(None, 5) == lbm.LBM_ERR_INVALID


@pytest.mark.parametrize("change", [
    {"dx": 0.0}, {"dt": float("nan")}, {"state": (0.0, 0.0, 0.0, 1.0)},
    {"state": (1.0, 0.0, 0.0, -1.0)}, {"rate": float("inf")}, {"k": float("nan")},
    {"nk": 0},
])
def test_vn_rejects_bad_arguments_on_host(change):
    from paper_0908_3749_gb300 import lbm
    state = change.get("state", (1.0, 0.1, 0.0, 1.0))
    rates = [1e4] * 16
    rates[6] = change.get("rate", 1e4)
    cases = lbm.vn_cases([state], [rates])
    k = np.zeros((0 if change.get("nk") == 0 else 2, 2))
    if k.shape[0]:
        k[1, 0] = change.get("k", 100.0)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_vn_spectrum(cases, k, change.get("dx", 1e-3), 1e-3, change.get("dt", 1e-5))
    assert ei.value.code == lbm.LBM_ERR_INVALID
    assert lbm.load().lbm_vn_last_error()


def test_probe_rejects_bad_arguments_on_host():
    """lbm_probe_fma_rate checks kind, output pointer and duration before it
    touches the device."""
    import ctypes
    from paper_0908_3749_gb300 import lbm
    lib = lbm.load()
    out = ctypes.c_double()
    for kind, millis, ptr in ((7, 50.0, ctypes.byref(out)), (-1, 50.0, ctypes.byref(out)),
                              (0, 0.5, ctypes.byref(out)), (1, 5000.0, ctypes.byref(out)),
                              (2, float("nan"), ctypes.byref(out)), (0, 50.0, None)):
        assert lib.lbm_probe_fma_rate(kind, millis, ptr, None) == lbm.LBM_ERR_INVALID


def test_eig16_rejects_empty_input():
    from paper_0908_3749_gb300 import lbm
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_eig16(np.zeros((0, 16, 16), complex))
    assert ei.value.code == lbm.LBM_ERR_INVALID


def _build_c_example(tmp_path):
    """Compiles tests/abi_example.c as C99 against include/ and links it to
    the library; returns (executable, environment)."""
    import shutil
    import subprocess
    from paper_0908_3749_gb300 import build, lbm
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lbm.load()
    exe = str(tmp_path / "abi_example")
    res = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                          "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_example.c"),
                          "-L", build.OUT, "-llbm", "-lm", "-o", exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=build.OUT + os.pathsep + os.environ.get("LD_LIBRARY_PATH", ""))
    return exe, env


def test_headers_are_c_and_a_c_program_links(tmp_path):
    """The ABI is plain C: a C99 program using only include/lbm.h compiles
    with -pedantic -Werror and links against the library. Without a GPU it
    must fail with an error status and a message, not crash."""
    import subprocess
    exe, env = _build_c_example(tmp_path)
    import torch
    if torch.cuda.is_available():
        return  # run by the GPU test
    res = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=60)
    assert res.returncode == 1 and "lbm_create failed" in res.stderr, (res.returncode, res.stderr)
