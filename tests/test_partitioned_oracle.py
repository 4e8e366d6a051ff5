"""The row-partitioned DCGS2 Arnoldi (oracle/partitioned.py) on 2 and 3 gloo ranks (CPU)
agrees with the sequential oracle, with exactly one all-reduce of 2k + 2 numbers per
step (plus three for the CGS2 finish): the partition the paper's distributed method uses,
checked without a second GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N_STEPS = 12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _operator():
    from synth import convdiff_csr
    return convdiff_csr(9, 3, [1.0, 0.5, 0.25]).to_scipy().tocsr()     # m = 729


def _worker(rank, P, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=P)
    from oracle.partitioned import dcgs2_arnoldi_rows
    from synth import gaussian_vector
    A = _operator()
    r0 = gaussian_vector(A.shape[0], 1002)
    calls = []

    def allreduce_sum(x):
        t = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64))
        dist.all_reduce(t)
        calls.append(t.numel())
        return t.numpy()

    def allgather(x):
        parts = [None] * P
        dist.all_gather_object(parts, x)
        return np.concatenate(parts)

    Q, H = dcgs2_arnoldi_rows(A, r0, N_STEPS, rank, P, allreduce_sum, allgather)
    out[rank] = (Q, H, calls)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("P", [2, 3])
def test_partitioned_dcgs2_matches_sequential_oracle(P):
    from oracle.arnoldi import dcgs2_arnoldi
    from oracle.partitioned import row_blocks
    from synth import gaussian_vector
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(P, _free_port(), out), nprocs=P, join=True)
    A = _operator()
    Qo, Ho = dcgs2_arnoldi(A, gaussian_vector(A.shape[0], 1002), N_STEPS)
    Q = np.vstack([out[p][0] for p in range(P)])
    for p in range(P):
        assert np.linalg.norm(out[p][1] - Ho) / np.linalg.norm(Ho) <= 1e-13    # replicated H
    assert np.abs(Q - Qo).max() <= 1e-12
    assert [b - a for a, b in row_blocks(A.shape[0], P)] == [out[p][0].shape[0] for p in range(P)]
    calls = out[0][2]
    assert calls[:N_STEPS] == [2 * k + 2 for k in range(N_STEPS)]   # one reduction per step
    assert len(calls) == N_STEPS + 3                                  # + C1, C2, ||u||
