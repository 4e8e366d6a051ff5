"""GPU parity of the row-partitioned DCGS2 step (dcgs2_part_reduce / dcgs2_part_update /
dcgs2_part_finish, Section 5's layout) against the FP64 oracle.

One GPU is available, so the ranks are emulated: (1) in one process, P ranks with their
own contexts and row blocks, whose partial sums are added on the device between the
launches (standing in for the all-reduce) and whose halos are copied from the other
ranks' vectors; (2) two processes on cuda:0 that exchange halos and sum partials through
gloo on the host between launches.  No kernel of one rank waits on another rank's.
Tolerances of the other DCGS2 parity tests: H 1e-12 relative, basis 1e-10 absolute."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_GRID, N_STEPS = 16, 30


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2104_01253_gb300 as kc
    return kc


def _operator():
    from synth import config2_operator
    return config2_operator(N_GRID)                    # m = 4096, 3D, Peclet 50


def _reference():
    from oracle import arnoldi as orc
    from synth import gaussian_vector
    Ah = _operator()
    r0 = gaussian_vector(Ah.m, 1002)
    Qo, Ho = orc.dcgs2_arnoldi(Ah.to_scipy(), r0, N_STEPS)
    return Ah, r0, Qo, Ho


def _rank_setup(kc, Ah, blocks, p):
    from paper_2104_01253_gb300 import partitioned as pt
    from synth import CSR
    lo, hi = blocks[p]
    rp, ci, va, glo, ghi = pt.local_rows(Ah.row_ptr, Ah.col_idx, Ah.val, lo, hi)
    A_local = kc.DeviceCSR(CSR(hi - lo, rp, ci, va))
    st = kc.ArnoldiState(hi - lo, N_STEPS + 1, kc.KC_F64)
    return A_local, st, glo, ghi


@pytest.mark.parametrize("mode", [1, 0])
@pytest.mark.parametrize("P", [2, 3])
def test_partitioned_step_emulated_ranks(kc, P, mode):
    from paper_2104_01253_gb300 import partitioned as pt
    Ah, r0, Qo, Ho = _reference()
    blocks = pt.row_blocks(Ah.m, P)
    ctxs = [kc.Context(0) for _ in range(P)]
    ranks = [_rank_setup(kc, Ah, blocks, p) for p in range(P)]
    for c in ctxs:
        c.set_fp64_mode(mode)
    n = N_STEPS
    for p, (A_l, st, _, _) in enumerate(ranks):
        lo, hi = blocks[p]
        kc.dcgs2_arnoldi_init(ctxs[p], A_l, st, torch.as_tensor(r0[lo:hi], device="cuda"))

    def w_ext(p):
        glo, ghi = ranks[p][2], ranks[p][3]
        parts = []
        for q, (lo, hi) in enumerate(blocks):
            a, b = max(lo, glo), min(hi, ghi)
            if a < b:
                parts.append(ranks[q][1].w[a - lo:b - lo])
        return torch.cat(parts)

    for k in range(n):
        partials = [torch.empty(2 * k + 2, dtype=torch.float64, device="cuda") for _ in range(P)]
        for p, (A_l, st, _, _) in enumerate(ranks):
            kc.dcgs2_part_reduce(ctxs[p], A_l, st, w_ext(p), partials[p])
        tot = torch.stack(partials).sum(0)               # the global sum of the step
        for p, (A_l, st, _, _) in enumerate(ranks):
            kc.dcgs2_part_update(ctxs[p], A_l, st, tot)
    tot = None
    for phase, size in ((0, n + 1), (1, n + 1), (2, 1), (3, 0)):
        partials = [torch.empty(max(size, 1), dtype=torch.float64, device="cuda")
                    for _ in range(P)]
        for p, (A_l, st, _, _) in enumerate(ranks):
            kc.dcgs2_part_finish(ctxs[p], A_l, st, phase, tot, partials[p] if size else None)
        tot = torch.stack(partials).sum(0) if size else None
    torch.cuda.synchronize()
    for c in ctxs:
        assert c.read_status() == 0
    Q = np.vstack([st.Q(n + 1).cpu().numpy() for _, st, _, _ in ranks])
    for _, st, _, _ in ranks:
        H = st.H(n + 1, n).cpu().numpy()
        assert np.linalg.norm(H - Ho) / np.linalg.norm(Ho) <= 1e-12
    assert np.abs(Q - Qo).max() <= 1e-10
    # the replicated H is the same on every rank, bit for bit
    H0 = ranks[0][1].H(n + 1, n).cpu().numpy()
    assert all(np.array_equal(H0, st.H(n + 1, n).cpu().numpy()) for _, st, _, _ in ranks)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, P, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=P)
    import paper_2104_01253_gb300 as kc
    from paper_2104_01253_gb300 import partitioned as pt
    from synth import gaussian_vector
    Ah = _operator()
    r0 = gaussian_vector(Ah.m, 1002)
    blocks = pt.row_blocks(Ah.m, P)
    ranges = [pt.local_rows(Ah.row_ptr, Ah.col_idx, Ah.val, lo, hi)[3:] for lo, hi in blocks]
    plans = [pt.halo_plan(blocks, p, glo, ghi) for p, (glo, ghi) in enumerate(ranges)]
    ctx = kc.Context(0)
    A_l, st, glo, ghi = _rank_setup(kc, Ah, blocks, rank)
    lo, hi = blocks[rank]
    sums = []

    def exchange(w_local):
        torch.cuda.synchronize()
        e = pt.halo_exchange(dist, blocks, rank, w_local.cpu(), glo, ghi, plans)
        return e.to("cuda")

    def allreduce(t):
        torch.cuda.synchronize()
        h = t.cpu()
        dist.all_reduce(h)
        sums.append(h.numel())
        return h.to("cuda")

    pt.expansion(kc, ctx, A_l, st, torch.as_tensor(r0[lo:hi], device="cuda"), N_STEPS,
                 exchange, allreduce)
    torch.cuda.synchronize()
    out[rank] = (st.Q(N_STEPS + 1).cpu().numpy(), st.H(N_STEPS + 1, N_STEPS).cpu().numpy(),
                 ctx.read_status(), sums)
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_step_two_processes_one_gpu(kc):
    """Two processes, each a rank with its own rows on cuda:0, through the package's
    driver (partitioned.expansion) with gloo on the host: one global sum of 2k + 2 numbers
    per step and three for the finish."""
    import torch.multiprocessing as mp
    P = 2
    Ah, r0, Qo, Ho = _reference()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(P, _free_port(), out), nprocs=P, join=True)
    Q = np.vstack([out[p][0] for p in range(P)])
    for p in range(P):
        assert out[p][2] == 0
        assert np.linalg.norm(out[p][1] - Ho) / np.linalg.norm(Ho) <= 1e-12
    assert np.abs(Q - Qo).max() <= 1e-10
    sums = out[0][3]
    assert sums[:N_STEPS] == [2 * k + 2 for k in range(N_STEPS)]
    assert sums[N_STEPS:] == [N_STEPS + 1, N_STEPS + 1, 1]
