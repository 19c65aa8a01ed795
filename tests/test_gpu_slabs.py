"""y-slab decomposition on the GPU: a run split into slab contexts (owned rows
plus ghost rows refreshed from the neighbours before every step) must advance
its owned rows exactly as the single-domain run: every field, psi(r, q) and the
stored populations bit for bit, over more than 20 steps, in FP64, FP32 and FP16
storage, on the fused path (whose tile-border fix-up then runs inside each
slab's extended rows) and on the two-pass path. Slabs in one process exchange
through device buffers; slabs in two processes (gloo, host buffers) share the
one GPU here, their kernels never waiting on each other. The single-domain run
is itself checked against the oracle (tests/test_gpu_parity.py); the FP64
slabs are also compared with the oracle directly at 1e-12."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FIELDS = ["rho_s", "psi_tot", "ux", "uy", "cxx", "cxy", "cyy", "thxx", "thxy", "thyy", "qrms",
          "vort"]


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available()
    from paper_2201_10132_gb300 import build, tfkt
    build.build()
    return tfkt


def _single(T, p, pert, steps):
    with T.Solver(p, pert) as s:
        s.step(steps)
        return s.moments(), s.psi(), s.populations()


def _run_slabs(T, p, pert, parts, steps):
    import torch
    from paper_2201_10132_gb300 import slabs as S
    slabs, bufs = [], []
    for y0, n in S.partition(p.ny, parts):
        s = T.Slab(p, y0, n, S.local_perturbation(pert, y0, n))
        nb = s.halo_bytes()
        slabs.append(s)
        bufs.append((torch.empty(nb, dtype=torch.uint8, device="cuda"),
                     torch.empty(nb, dtype=torch.uint8, device="cuda")))
    # every context runs on the legacy default stream: packs, unpacks and steps are ordered
    S.exchange_local(slabs, bufs)
    for _ in range(steps):
        for s in slabs:
            s.step(1)
        S.exchange_local(slabs, bufs)
    f = [s.moments() for s in slabs]
    fields = {k: np.concatenate([s.owned(fk[k]) for s, fk in zip(slabs, f)]) for k in FIELDS}
    psi = np.concatenate([s.owned(s.psi(), axis=0) for s in slabs])
    pops = np.concatenate([s.owned(s.populations()) for s in slabs], axis=1)
    kinds = [s.info for s in slabs]
    for s in slabs:
        s.close()
    return fields, psi, pops, kinds


# nx, ny, slabs, precision, steps[, stress quasi-equilibrium]; S = 6, R = 3 (32 Q-nodes)
CASES = [
    (64, 48, 2, "FP64", 24),     # fused path (tile multiples), two slabs of 24 rows
    (64, 64, 3, "FP64", 21),     # fused, uneven slabs 24 / 24 / 16
    (70, 40, 2, "FP64", 22),     # two-pass path (nx not a multiple of 32)
    (70, 45, 3, "FP64", 22),     # two-pass, slabs of 15 rows (not multiples of 8)
    (64, 48, 2, "FP32", 24),
    (64, 48, 3, "FP16", 22),
    (64, 48, 2, "FP64", 22, True),   # the stress quasi-equilibrium on the fused path
]


def _params(T, nx, ny, prec, stress=False):
    if stress:      # momentum relaxation time below 3 beta nu, as the stress model requires
        return T.Params(nx, ny, 6, 3.0, 5.0, 2.0, 0.5, 0.05, 1, 0.03, 0.0, 1, getattr(T, prec),
                        0.0, T.QE_STRESS)
    return T.Params(nx, ny, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, ic_mode=1, precision=getattr(T, prec))


@pytest.mark.parametrize("case", CASES)
def test_slabs_in_one_process_are_bit_identical(T, oracle_mod, case):
    from paper_2201_10132_gb300.inputs import perturbation
    nx, ny, parts, prec, steps = case[:5]
    stress = len(case) > 5 and case[5]
    p = _params(T, nx, ny, prec, stress)
    pert = perturbation(nx, ny, 9, 0.05, 0.05)
    ref, ref_psi, ref_pops = _single(T, p, pert, steps)
    got, psi, pops, _ = _run_slabs(T, p, pert, parts, steps)
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k], equal_nan=True), k
    assert np.array_equal(psi, ref_psi)
    assert np.array_equal(pops, ref_pops)
    if prec == "FP64":
        lat = (oracle_mod.map_params(nx, ny, 6, 3.0, 5.0, 2.0, 0.5, 0.05, 1, 0.03, 0.0, 0.0, 1)
               if stress else oracle_mod.map_params(nx, ny, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1))
        o = oracle_mod.Oracle(lat)
        o.init(pert, 1)
        o.step(steps)
        f = o.fields()
        for k in FIELDS:
            assert np.abs(got[k] - f[k]).max() <= 1e-12 * np.abs(f[k]).max(), k


def test_slab_rows_and_errors(T):
    p = T.Params(64, 48, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, precision=T.FP64)
    with T.Slab(p, 24, 24) as s:
        assert s.rows() == (24, 24, T.SLAB_GHOST)
        assert s.info["ny"] == 24 + 2 * T.SLAB_GHOST
        with pytest.raises(T.TfktError):
            s.pack(T.SLAB_HIGH, 0, s.halo_bytes(), True)          # NULL buffer
        with pytest.raises(T.TfktError):
            s.pack(2, 1, s.halo_bytes(), True)                     # unknown side
        # a device message must start on a 16-byte boundary (checked before any launch)
        import torch
        nb = s.halo_bytes()
        buf = torch.zeros(nb + 16, dtype=torch.uint8, device="cuda")
        with pytest.raises(T.TfktError) as e:
            s.pack(T.SLAB_LOW, buf.data_ptr() + 8, nb, True)
        assert e.value.status == T.EINVAL
        s.pack(T.SLAB_LOW, buf.data_ptr(), nb, True)               # the context is still usable
        s.unpack(T.SLAB_HIGH, buf.data_ptr(), nb, True)
        s.step(1)
    import ctypes
    with T.Solver(p) as s:                                         # not a slab context
        n = ctypes.c_size_t()
        assert T.lib().tfkt_slab_halo_bytes(s._h, ctypes.byref(n)) == 1
    for bad in ((0, 7), (48, 8), (-1, 8)):
        with pytest.raises(T.TfktError):
            T.Slab(p, *bad)
    # the learned block reaches further than one step: not on a slab
    q = T.Params(64, 48, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1, precision=T.FP32)
    with T.Slab(q, 0, 24) as s:
        with pytest.raises(T.TfktError) as e:
            T.lpm_run(s, None, 1, K=4, mode=T.LPM_FROZEN)
        assert e.value.status == 1


def _rank_run(rank, world, port, case, out):
    import torch
    import torch.distributed as dist
    from paper_2201_10132_gb300 import slabs as S, tfkt as T
    from paper_2201_10132_gb300.inputs import perturbation
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    nx, ny, steps = case
    p = T.Params(nx, ny, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, ic_mode=1, precision=T.FP64)
    pert = perturbation(nx, ny, 9, 0.05, 0.05)
    y0, n = S.partition(ny, world)[rank]
    s = T.Slab(p, y0, n, S.local_perturbation(pert, y0, n))
    nb = s.halo_bytes()
    send = [torch.zeros(nb, dtype=torch.uint8).pin_memory() for _ in range(2)]
    recv = [torch.zeros(nb, dtype=torch.uint8).pin_memory() for _ in range(2)]
    pack = lambda side, t: s.pack(side, t.data_ptr(), nb, False)
    unpack = lambda side, t: s.unpack(side, t.data_ptr(), nb, False)
    S.exchange_ranks(pack, unpack, send, recv, dist, rank, world)
    for _ in range(steps):
        s.step(1)
        S.exchange_ranks(pack, unpack, send, recv, dist, rank, world)
    mine = np.stack([s.owned(s.moments()[k]) for k in FIELDS])
    s.close()
    np.save(f"{out}.{rank}.npy", mine)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_slabs_in_two_processes_with_host_exchange(T, tmp_path):
    """Two gloo ranks, each a slab on this GPU, exchanging host copies of the
    ghost rows (the path a multi-GPU run takes with host-staged messages)."""
    import torch.multiprocessing as mp
    from paper_2201_10132_gb300.inputs import perturbation
    case = (64, 48, 22)
    out = str(tmp_path / "slab")
    mp.spawn(_rank_run, args=(2, _free_port(), case, out), nprocs=2, join=True)
    got = np.concatenate([np.load(f"{out}.{r}.npy") for r in range(2)], axis=1)
    nx, ny, steps = case
    p = T.Params(nx, ny, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, ic_mode=1, precision=T.FP64)
    ref, _, _ = _single(T, p, perturbation(nx, ny, 9, 0.05, 0.05), steps)
    for i, k in enumerate(FIELDS):
        assert np.array_equal(got[i], ref[k]), k
