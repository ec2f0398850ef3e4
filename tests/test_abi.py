"""The C ABI library builds, loads without a GPU and exports every entry
point include/dgsm.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dgsm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path():
    names = _declared()
    for must in ("dgsm_build", "dgsm_attenuate", "sh_fit", "sh_relight", "dgsm_bin"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2601_01660_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_without_gpu():
    from paper_2601_01660_b300 import native
    nat = native()
    p = nat.Params.make()
    assert (p.kappa, p.tile, p.chunk, p.atlas_dtype) == (1.0, 8, 128, 0)
    assert abs(p.eps_cull - 1e-7) < 1e-12
    rp = nat.RelightParams()
    nat._lib.dgsm_default_relight_params(ctypes.byref(rp))
    assert (rp.q, rp.gamma, rp.t_max, rp.n_theta, rp.n_phi) == (1.0, 1.0, 10.0, 32, 64)
    assert nat._lib.dgsm_status_string(6) == b"normal equations not positive definite"
