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
    assert st == 1 and b"null" in L.ipc_last_error() or b"bad" in L.ipc_last_error()


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
