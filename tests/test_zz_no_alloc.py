"""tfkt_moments_noalloc against tfkt_moments, through the C-ABI.

tfkt_moments_noalloc serves callers that may not allocate device memory where
they need the fields (a fixed memory arena, or a host framework whose
allocator cannot be entered there): its scratch is a static device array of
the library. It must return the same fields as a context's tfkt_moments on the
same state, on consecutive calls that reuse the array, and must reject a grid
whose scratch would not fit. The file is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _align(v, a=256):
    return (v + a - 1) // a * a


@pytest.mark.parametrize("fp64", [True, False])
def test_noalloc_matches_moments_on_two_calls(fp64):
    import torch
    from paper_2201_10132_gb300 import build, tfkt
    from paper_2201_10132_gb300.inputs import perturbation
    build.build()
    nx, ny = 70, 40
    prec = tfkt.FP64 if fp64 else tfkt.FP32
    esz = 8 if fp64 else 4
    p = tfkt.Params(nx, ny, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, ic_mode=1, precision=prec)
    ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
    names = tfkt.FIELDS
    mask = tfkt.field_mask(names)
    with tfkt.Solver(p, perturbation(nx, ny, 5, 0.05, 0.05), workspace=ws) as s:
        npl = 9 + 25 * s.info["nq"]
        buf_bytes = _align(npl * ny * s.info["pitch"] * esz)
        for call in range(2):
            s.step(3 + call)
            n = s.get_info()["step"]
            ref = torch.empty((len(names), ny, nx), dtype=torch.float64, device="cuda")
            s.moments(names, out=ref)
            got = torch.full_like(ref, float("nan"))
            tfkt.moments_noalloc(p, ws.data_ptr() + (n % 2) * buf_bytes, mask, got.data_ptr(),
                                 got.numel() * 8)
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            assert np.isfinite(g).all()
            uscale = np.abs(r[2:4]).max()
            for k, name in enumerate(names):
                scale = uscale if name in ("ux", "uy", "vort") else np.abs(r[k]).max()
                err = np.abs(g[k] - r[k]).max() / scale
                assert err < (1e-12 if fp64 else 2e-5), (call, name, err)


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
