"""The C ABI library builds for sm_103a, loads, and exports every function include/ipc.h
declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import subprocess

from paper_2503_05020_b300 import build as B
from paper_2503_05020_b300 import ipc


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    names = ipc.declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in names:
        assert f" T {n}" in out, n


def test_version_and_error_strings_without_gpu():
    L = ipc.lib()
    assert b"sm_103a" in L.ipc_version()
    # a null scene is rejected on the host before any CUDA call
    st = L.ipc_step(None, 1)
    err = L.ipc_last_error()
    assert st == 1 and (b"null" in err or b"bad" in err)


def test_env_validation_on_host():
    """Inverted rest tets and empty environments are rejected on the host."""
    import numpy as np
    from paper_2503_05020_b300 import scenes as S

    env = S.single_tet_env()
    env["soft"][0]["tets"] = env["soft"][0]["tets"][:, [0, 2, 1, 3]].copy()
    try:
        ipc.estimate_bytes(env)
        raise AssertionError("inverted tet accepted")
    except ipc.IpcError as e:
        assert e.status == 6
    ok = S.cube_squeeze_env(0)
    assert ipc.estimate_bytes(ok) > 100_000


def test_gravity_codes_are_validated_on_host():
    """Per-step gravity codes 0..7 are accepted (none, the scene's vector, the six axis
    phases); other values are rejected before anything reaches the GPU."""
    import numpy as np
    from paper_2503_05020_b300 import scenes as S

    env = S.single_tet_env(n_steps=3)
    env["gravity"] = np.array([0, 1, 7], dtype=np.uint8)
    assert ipc.estimate_bytes(env) > 0
    env["gravity"] = np.array([0, 7, 8], dtype=np.uint8)
    try:
        ipc.estimate_bytes(env)
        raise AssertionError("gravity code 8 accepted")
    except ipc.IpcError as e:
        assert e.status == 1


def _rejected(fn, status):
    try:
        fn()
    except ipc.IpcError as e:
        assert e.status == status, (e.status, e)
        return str(e)
    raise AssertionError("accepted")


def test_scene_parameters_are_validated_on_host():
    """A scene with a non-positive time step, contact distance or stiffness, an unknown
    precision or an unsupported cluster size is rejected (IPC_ERR_ARG) before any CUDA call."""
    from paper_2503_05020_b300 import scenes as S

    good = S.scene_params(0.01)
    for key, bad in (("dt", 0.0), ("dhat", -1e-3), ("kappa", 0.0), ("dt", float("nan"))):
        _rejected(lambda: ipc.Scene(dict(good, **{key: bad})), 1)
    _rejected(lambda: ipc.Scene(good, precision=5), 1)
    _rejected(lambda: ipc.Scene(good, pcg_cluster=3), 1)


def test_env_meshes_are_validated_on_host():
    """Out-of-range tet and triangle indices, an empty soft body, an affine surface that encloses
    no volume (triangles turned inward) and an empty schedule are rejected on the host."""
    import numpy as np
    from paper_2503_05020_b300 import scenes as S

    env = S.single_tet_env(n_steps=2)
    env["soft"][0]["tets"] = np.array([[0, 1, 2, 4]], dtype=np.int32)
    assert "tet index" in _rejected(lambda: ipc.estimate_bytes(env), 1)

    env = S.single_tet_env(n_steps=2)
    env["soft"][0]["tris"] = np.array([[0, 1, 9]], dtype=np.int32)
    assert "triangle index" in _rejected(lambda: ipc.estimate_bytes(env), 1)

    env = S.resting_env("rigid", n_steps=2)
    env["affine"][0]["tris"] = env["affine"][0]["tris"][:, [0, 2, 1]].copy()
    assert "volume" in _rejected(lambda: ipc.estimate_bytes(env), 1)

    env = S.resting_env("rigid", n_steps=2)
    env["gravity"] = env["gravity"][:0]
    env["targets"] = env["targets"][:0]
    _rejected(lambda: ipc.estimate_bytes(env), 1)

    env = S.single_tet_env(n_steps=2)
    env["soft"][0]["tets"] = env["soft"][0]["tets"][:0]
    assert "empty" in _rejected(lambda: ipc.estimate_bytes(env), 1)


def test_product_path_has_no_cpu_fallback():
    """The package never reaches the oracle (no import of it anywhere in the product modules),
    and the binding fails loudly, instead of falling back to anything, when the library is
    missing."""
    import ast
    import importlib

    pkg = os.path.dirname(ipc.__file__)
    for name in os.listdir(pkg):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, name)).read())
        for node in ast.walk(tree):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (name, mods)

    fresh = importlib.import_module("paper_2503_05020_b300.ipc")
    saved_path, saved_lib = fresh.LIB_PATH, fresh._lib
    try:
        fresh.LIB_PATH, fresh._lib = os.path.join(pkg, "missing", "libipc_b300.so"), None
        try:
            fresh.lib()
            raise AssertionError("missing library did not raise")
        except ImportError as e:
            assert "not built" in str(e)
    finally:
        fresh.LIB_PATH, fresh._lib = saved_path, saved_lib


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every descriptor struct of the binding has the size and field offsets the C compiler gives
    include/ipc.h (a layout mismatch would pass garbage through the ABI)."""
    import ctypes as C

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"ipc_scene_desc": ipc.SceneDesc, "ipc_soft_body_desc": ipc.SoftDesc,
               "ipc_affine_body_desc": ipc.AffineDesc, "ipc_joint_desc": ipc.JointDesc, "ipc_env_desc": ipc.EnvDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ipc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_joint_descriptors_are_validated_on_host():
    """A joint must join two distinct affine bodies of its env with a positive stiffness."""
    from paper_2503_05020_b300 import scenes as S

    env = S.pendulum_env()
    assert ipc.estimate_bytes(env) > 0
    for bad in (dict(b=2), dict(b=0), dict(k=0.0), dict(a=-1)):
        e = dict(env, joints=[dict(env["joints"][0], **bad)])
        try:
            ipc.estimate_bytes(e)
            raise AssertionError(f"bad joint accepted: {bad}")
        except ipc.IpcError as err:
            assert err.status == 1
