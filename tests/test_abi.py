"""C-ABI checks that need no GPU: the library loads, exports every function that
include/*.h declares, and rejects invalid parameters before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    from paper_2201_10132_gb300 import build, tfkt
    build.build()
    return tfkt


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(tfkt_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(T):
    names = _declared()
    assert {"tfkt_create", "tfkt_step", "tfkt_moments", "tfkt_destroy", "tfkt_mlp_forward",
            "tfkt_mlp_loss_grad", "tfkt_lpm_run"} <= set(names)
    lib = ctypes.CDLL(T.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("header", ["tfkt.h", "tfkt_lpm.h"])
def test_headers_are_plain_c(header, tmp_path):
    """The boundary's headers compile on their own as strict C99 (no torch or C++
    types in the interface) and as C++."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text(f'#include "{header}"\n')
    inc = os.path.join(ROOT, "include")
    for cmd in (["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only"],
                ["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-x", "c++"]):
        r = subprocess.run(cmd + ["-I", inc, str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_every_status_has_a_name(T):
    """The statuses of include/tfkt.h, the binding's names and tfkt_status_string
    agree; an unknown code has its own text."""
    lib = ctypes.CDLL(T.LIB_PATH)
    lib.tfkt_status_string.restype = ctypes.c_char_p
    lib.tfkt_status_string.argtypes = [ctypes.c_int]
    hdr = open(os.path.join(ROOT, "include", "tfkt.h")).read()
    codes = {int(v): n for n, v in re.findall(r"\b(TFKT_[A-Z]+) = (\d+)", hdr)}
    assert codes == T.STATUS
    texts = {lib.tfkt_status_string(c).decode() for c in codes}
    assert len(texts) == len(codes) and "unknown status" not in texts
    assert lib.tfkt_status_string(99).decode() == "unknown status"
    assert T.ETIMEOUT == 7 and codes[T.ETIMEOUT] == "TFKT_ETIMEOUT"


def test_lattice_order_is_a_velocity_set(T):
    import numpy as np
    c9, c25 = T.lattice()
    assert len({tuple(v) for v in c9.tolist()}) == 9
    assert len({tuple(v) for v in c25.tolist()}) == 25
    assert all((np.abs(v) <= 1).all() for v in c25)
    assert sorted(int((v != 0).sum()) for v in c25) == [0] + [2] * 24


def test_required_bytes_matches_layout(T):
    p = T.Params(4096, 4096, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 64, precision=T.FP32)
    n = T.required_bytes(p)
    nodes = 4096 * 4096
    pops = (9 + 25 * 32) * nodes * 4 * 2
    assert pops < n < pops * 1.1


@pytest.mark.parametrize("kw", [dict(beta=0.0), dict(beta=1.5), dict(re=0.0), dict(u0=0.5),
                                dict(wi=0.0), dict(tau2=1e-4), dict(q_radius=0.0), dict(nx=0),
                                dict(q_side=65), dict(precision=7), dict(ic_mode=3),
                                dict(q_radius=0.1, q_side=2), dict(fene_b=-1.0),
                                dict(fene_b=25.0)])  # the disk reaches past Q0
def test_invalid_parameters(T, kw):
    args = dict(nx=8, ny=8, q_side=4, q_radius=2.0, re=5.0, wi=0.5, beta=0.2)
    args.update(kw)
    with pytest.raises(T.TfktError) as e:
        T.required_bytes(T.Params(**args))
    assert e.value.status == 1  # TFKT_EINVAL


def test_fene_disk_inside_q0_is_accepted(T, oracle_mod):
    """The library's FENE bound on the disk is the oracle's (R < Q0 = sqrt(b sigma_Q^2))."""
    lat = oracle_mod.map_params(64, 64, 8, 4.0, 5.0, 0.5, 0.2, 0.05, 1, fene_b=25.0)
    q0 = (25.0 * lat.sigma_q2) ** 0.5
    T.required_bytes(T.Params(64, 64, 8, 4.0, 5.0, 0.5, 0.2, fene_b=25.0))
    T.required_bytes(T.Params(64, 64, 8, 0.999 * q0, 5.0, 0.5, 0.2, fene_b=25.0))
    with pytest.raises(T.TfktError):
        T.required_bytes(T.Params(64, 64, 8, 1.001 * q0, 5.0, 0.5, 0.2, fene_b=25.0))


def test_fp16_population_buffer_layout(T):
    """FP16 storage keeps 9 + 25 nq plane slots of half and the nine solvent planes
    as floats after them (include/tfkt.h): against FP32 storage each of the two
    population buffers is 2 bytes per slot smaller and 9 x 4 bytes per node larger;
    everything else in the workspace (float moment planes, tables) is the same."""
    base = dict(nx=1024, ny=1024, q_side=6, q_radius=3.0, re=10.0, wi=1.0, beta=0.2, u0=0.05,
                k_periods=16)
    p32 = T.required_bytes(T.Params(**base, precision=T.FP32))
    p16 = T.required_bytes(T.Params(**base, precision=T.FP16))
    plane = 1024 * 1024            # pitch 1024: planes are multiples of 256 bytes
    npl = 9 + 25 * 32
    assert p32 - p16 == 2 * (npl * plane * 2 - 9 * plane * 4)
