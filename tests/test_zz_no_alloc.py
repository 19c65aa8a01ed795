"""tfkt_moments_noalloc against tfkt_moments, through the C-ABI.

tfkt_moments_noalloc serves callers that may not allocate device memory where
they need the fields (a fixed memory arena, or a host framework whose
allocator cannot be entered there): its scratch is a static device array of
the library. It must return the same fields as a context's tfkt_moments on the
same state, on consecutive calls that reuse the array (also when calls for
another run, with other lattice tables, come in between), in every storage
precision, and must reject a grid whose scratch would not fit. The file is
named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# the storage precision's parity tolerance against the oracle (tests/test_gpu_parity.py);
# both entry points compute the fields in the same precision from the same state
TOL = {"FP64": 1e-12, "FP32": 2e-5, "FP16": 2e-5}


def _align(v, a=256):
    return (v + a - 1) // a * a


def _buffer_bytes(info, nx, ny, storage):
    """One population buffer of a context: (9 + 25 nq) planes of the storage type,
    plus, under FP16 storage, the nine solvent planes as floats after them;
    rounded up to 256 and never less than the field staging size."""
    npl = 9 + 25 * info["nq"]
    plane = ny * info["pitch"]
    esz = {"FP64": 8, "FP32": 4, "FP16": 2}[storage]
    b = npl * plane * esz + (9 * plane * 4 if storage == "FP16" else 0)
    return _align(max(b, 12 * nx * ny * 8))


def _compare(got, ref, names, tol, what):
    uscale = max(np.abs(ref[names.index("ux")]).max(), np.abs(ref[names.index("uy")]).max())
    assert np.isfinite(got).all(), what
    for k, name in enumerate(names):
        scale = uscale if name in ("ux", "uy", "vort") else np.abs(ref[k]).max()
        err = np.abs(got[k] - ref[k]).max() / scale
        assert err < tol, (what, name, err)


def _noalloc(tfkt, p, ptr, mask, shape):
    """The fields of mask, in increasing bit order, from the population buffer at ptr."""
    import torch
    got = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    tfkt.moments_noalloc(p, ptr, mask, got.data_ptr(), got.numel() * 8)
    torch.cuda.synchronize()
    return got.cpu().numpy()


@pytest.mark.parametrize("storage", ["FP64", "FP32", "FP16"])
def test_noalloc_matches_moments_on_two_calls(storage):
    import torch
    from paper_2201_10132_gb300 import build, tfkt
    from paper_2201_10132_gb300.inputs import perturbation
    build.build()
    nx, ny = 70, 40
    p = tfkt.Params(nx, ny, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, ic_mode=1,
                    precision=getattr(tfkt, storage))
    ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
    names = tfkt.FIELDS
    mask = tfkt.field_mask(names)
    with tfkt.Solver(p, perturbation(nx, ny, 5, 0.05, 0.05), workspace=ws) as s:
        buf_bytes = _buffer_bytes(s.info, nx, ny, storage)
        for call in range(2):
            s.step(3 + call)
            n = s.get_info()["step"]
            ref = s.moments(names)
            r = np.stack([ref[k] for k in names])
            g = _noalloc(tfkt, p, ws.data_ptr() + (n % 2) * buf_bytes, mask, r.shape)
            _compare(g, r, names, TOL[storage], call)


def test_noalloc_alternating_runs_reuse_or_refresh_tables():
    """Two runs with different grids and parameters, called in the order A, B, A, A:
    each call must use its own run's lattice tables, whether the array holds them
    from the previous call or not."""
    import torch
    from paper_2201_10132_gb300 import build, tfkt
    from paper_2201_10132_gb300.inputs import perturbation
    build.build()
    runs = [(tfkt.Params(64, 32, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, ic_mode=1, precision=tfkt.FP32),
             perturbation(64, 32, 1, 0.05, 0.05)),
            (tfkt.Params(40, 24, 8, 4.0, 3.0, 1.0, 0.5, 0.05, 2, ic_mode=0, precision=tfkt.FP32),
             perturbation(40, 24, 2, 0.05, 0.05))]
    names = ["rho_s", "ux", "uy", "cxx", "cxy", "thyy", "vort"]
    mask = tfkt.field_mask(names)
    sols, wss, refs, ptrs = [], [], [], []
    for p, pert in runs:
        ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
        s = tfkt.Solver(p, pert, workspace=ws)
        s.step(5)
        ref = s.moments(names)
        refs.append(np.stack([ref[k] for k in names]))
        ptrs.append(ws.data_ptr() + 1 * _buffer_bytes(s.info, p.nx, p.ny, "FP32"))
        sols.append(s)
        wss.append(ws)
    for i in (0, 1, 0, 0):
        g = _noalloc(tfkt, runs[i][0], ptrs[i], mask, refs[i].shape)
        _compare(g, refs[i], names, TOL["FP32"], i)
    for s in sols:
        s.close()


def test_noalloc_after_learned_block():
    """A learned block leaves its polymer increment pending; the population buffer
    holds the complete state once tfkt_populations has added it."""
    import torch
    from paper_2201_10132_gb300 import build, tfkt, train_lpm
    from paper_2201_10132_gb300.inputs import perturbation
    build.build()
    nx, ny = 64, 32
    p = tfkt.Params(nx, ny, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1, ic_mode=1, precision=tfkt.FP32)
    ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
    names = ["psi_tot", "ux", "uy", "cxx", "cxy", "cyy"]    # the output's order: bit order
    mask = tfkt.field_mask(names)
    vec, _ = train_lpm.load()
    net = tfkt.Mlp(vec)
    with tfkt.Solver(p, perturbation(nx, ny, 4, 0.05, 0.05), workspace=ws) as s:
        s.step(40)
        tfkt.lpm_run(s, net, 1, K=8, tile=16, threshold=1e9)
        n = s.get_info()["step"]
        assert n == 49
        s.populations()          # adds the pending increment to the stored populations
        ref = s.moments(names)
        r = np.stack([ref[k] for k in names])
        ptr = ws.data_ptr() + (n % 2) * _buffer_bytes(s.info, nx, ny, "FP32")
        g = _noalloc(tfkt, p, ptr, mask, r.shape)
        _compare(g, r, names, TOL["FP32"], "after flush")
    net.close()


def test_noalloc_rejects_grid_beyond_scratch():
    import torch
    from paper_2201_10132_gb300 import build, tfkt
    build.build()
    p = tfkt.Params(1024, 1024, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, precision=tfkt.FP32)
    dst = torch.empty((1024, 1024), dtype=torch.float64, device="cuda")
    pops = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(tfkt.TfktError) as e:
        tfkt.moments_noalloc(p, pops.data_ptr(), tfkt.field_mask(["ux"]), dst.data_ptr(),
                             dst.numel() * 8)
    assert e.value.status == 1 and "scratch" in str(e.value)
